// sve_batch.cu -- many independent runs of the step in one pair of launches
// per step (include/sve.h, sve_batch_*).
//
// Every run keeps its own grid, parameters, CFL time step, time and mass
// sums.  Work is cut into tiles of NT interfaces (or cells) of one run; a
// tile table lists the tiles of all runs in a schedule order, and each
// launch covers the whole table, so runs of uneven size share the GPU
// without one launch per run.  Each run's last tile to finish (an atomic
// ticket per run, no waiting) turns that run's per-tile partials into its
// time step (interface launch) or its mass sums and time (cell launch).  The
// per-interface and per-cell arithmetic is the single-run code
// (interface_item, cell_item of sve_device.cuh), so every run of a batch
// steps as it would alone, up to the compiler's FMA contraction choices in
// these separately compiled kernels (round-off level).  Tile size and schedule are picked by
// sve_batch_autotune from timed trial steps.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/sve.h"
#include "sve_device.cuh"

using sve::DevParams;
using sve::DevScalars;
using sve::DevState;

namespace {

template <typename T>
struct BatchRun {
  DevParams P;
  DevState<T> S;
  int part_if;    // first interface partial (2 doubles each) of this run
  int ntile_if;   // interface tiles of this run (at the current tile size)
  int part_cell;  // first cell partial
  int ntile_cell;
};

// Copy the run record of the block's tile into shared memory.
template <typename T>
__device__ __forceinline__ void load_run(const BatchRun<T>* runs, int r, BatchRun<T>* dst) {
  const int* src = (const int*)(runs + r);
  int* d = (int*)dst;
  for (int w = threadIdx.x; w < (int)(sizeof(BatchRun<T>) / sizeof(int)); w += blockDim.x) d[w] = src[w];
  __syncthreads();
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT) batch_interface_kernel(const BatchRun<T>* runs, const int2* tiles,
                                                             DevScalars* sc, double* spart) {
  __shared__ BatchRun<T> R;
  __shared__ bool last;
  __shared__ double sh[2 * (NT / 32)];
  const int2 t = tiles[blockIdx.x];
  load_run(runs, t.x, &R);
  const DevParams& P = R.P;
  const long long item = (long long)t.y * NT + threadIdx.x;
  double sx = 0.0, sy = 0.0;
  int iters = 0;
  bool fail = false;
  if (item < P.nfx) {
    fail = !sve::interface_item(P, R.S, false, item, sx, iters);
  } else if (item < P.nfx + P.nfy) {
    fail = !sve::interface_item(P, R.S, true, item - P.nfx, sy, iters);
  }
  if (fail) atomicOr(&sc[t.x].status, sve::ST_RIEMANN);
  int dummy = 0;
  sve::block_maxbits_sum<NT>(sx, iters);
  sve::block_maxbits_sum<NT>(sy, dummy);
  if (threadIdx.x == 0) {
    atomicAdd(&sc[t.x].newton_iters, (unsigned long long)iters);
    spart[2 * (R.part_if + t.y)] = sx;
    spart[2 * (R.part_if + t.y) + 1] = sy;
    __threadfence();
    const unsigned int ticket = atomicAdd(&sc[t.x].done_iface, 1u);
    last = (ticket == (unsigned)R.ntile_if - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // L2 loads after the fence; integer max of the bit patterns of the
  // non-negative speeds
  const long long* bp = reinterpret_cast<const long long*>(spart) + 2 * (size_t)R.part_if;
  long long bx = 0, by = 0;
#pragma unroll 4
  for (int b = threadIdx.x; b < R.ntile_if; b += NT) {
    bx = max(bx, __ldcg(bp + 2 * b));
    by = max(by, __ldcg(bp + 2 * b + 1));
  }
  double mx = __longlong_as_double(bx), my = __longlong_as_double(by);
  mx = sve::block_max<NT>(mx, sh);
  my = sve::block_max<NT>(my, sh);
  if (threadIdx.x == 0) {
    double dt = (P.dim == 1) ? P.cfl * P.dx / mx : P.cfl / (mx / P.dx + my / P.dy);
    if (!(dt > 0.0) || !isfinite(dt)) { atomicOr(&sc[t.x].status, sve::ST_DT); dt = 0.0; }
    sc[t.x].dt = dt;
    sc[t.x].Sx = mx;
    sc[t.x].Sy = my;
    sc[t.x].done_iface = 0u;
  }
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT) batch_cell_kernel(const BatchRun<T>* runs, const int2* tiles, DevScalars* sc,
                                                        double* mpart) {
  __shared__ BatchRun<T> R;
  __shared__ bool last;
  __shared__ double sh[2 * (NT / 32)];
  const int2 t = tiles[blockIdx.x];
  load_run(runs, t.x, &R);
  const DevParams& P = R.P;
  const long long k = (long long)t.y * NT + threadIdx.x;
  double mh = 0.0, mz = 0.0;
  if (k < (long long)P.nx * P.ny) {
    const int st = sve::cell_item(P, R.S, k, sc[t.x].dt, mh, mz);
    if (st) atomicOr(&sc[t.x].status, st);
  }
  sve::block_sum2<NT>(mh, mz, sh);
  if (threadIdx.x == 0) {
    mpart[2 * (R.part_cell + t.y)] = mh;
    mpart[2 * (R.part_cell + t.y) + 1] = mz;
    __threadfence();
    const unsigned int ticket = atomicAdd(&sc[t.x].done_cell, 1u);
    last = (ticket == (unsigned)R.ntile_cell - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double a, b;
  sve::reduce_partials<NT>(mpart + 2 * R.part_cell, (unsigned)R.ntile_cell, a, b, sh);
  if (threadIdx.x == 0) {
    const double cell = P.dx * (P.dim == 2 ? P.dy : 1.0);
    sc[t.x].mass_h = a * cell;
    sc[t.x].mass_z = b * cell;
    sc[t.x].t += sc[t.x].dt;
    sc[t.x].steps += 1;
    sc[t.x].done_cell = 0u;
  }
}

constexpr int kBatchGraphSteps = 8;
constexpr int kTileSizes[2] = {128, 256};
constexpr int kSchedules = 2;  // 0: run after run (largest first), 1: round robin over runs

}  // namespace

__attribute__((visibility("hidden"))) int sve_internal_validate(const sve_config* c);
__attribute__((visibility("hidden"))) void sve_internal_make_params(const sve_config* c, DevParams* P);

struct sve_batch {
  int nruns = 0;
  int precision = SVE_FP64;
  size_t elem = 8;
  std::vector<DevParams> P;
  std::vector<long long> next;       // padded cells per run
  std::vector<size_t> off;           // byte offset of each run's block in the arena
  std::vector<int> has_state;
  void* arena = nullptr;
  size_t arena_bytes = 0;
  void* d_runs = nullptr;            // BatchRun<T>[nruns]
  int2* d_tiles_if = nullptr;
  int2* d_tiles_cell = nullptr;
  int nt_if = 0, nt_cell = 0;
  DevScalars* d_sc = nullptr;
  double* d_spart = nullptr;
  double* d_mpart = nullptr;
  double* d_init_part = nullptr;     // partials for the per-run init kernel
  int tile = 256, schedule = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t capture = nullptr;
  cudaGraphExec_t graph = nullptr;
  long long last_launches = 0;
};

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Field f (0..12) and fluctuation planes of run r inside the arena.
size_t run_bytes(const DevParams& P, size_t elem) {
  const size_t next = (size_t)(P.nx + 2) * (size_t)(P.ny + 2);
  return 13 * align256(elem * next) + align256(8 * elem * (size_t)P.nfx) +
         align256(8 * elem * (size_t)(P.nfy > 0 ? P.nfy : 1));
}

template <typename T>
DevState<T> run_state(const sve_batch* b, int r) {
  DevState<T> S;
  const DevParams& P = b->P[r];
  const size_t next = (size_t)(P.nx + 2) * (size_t)(P.ny + 2);
  char* base = (char*)b->arena + b->off[r];
  T** f[13] = {&S.h, &S.hu, &S.hv, &S.z, &S.tau, &S.u, &S.v, &S.pi, &S.omx, &S.omy, &S.ca, &S.cbx, &S.cby};
  for (int k = 0; k < 13; ++k) { *f[k] = (T*)base; base += align256(b->elem * next); }
  S.fx = (T*)base;
  base += align256(8 * b->elem * (size_t)P.nfx);
  S.fy = (T*)base;
  return S;
}

long long tiles_of(long long items, int tile) { return (items + tile - 1) / tile; }

// Build the run records and tile tables for a tile size and schedule.
template <typename T>
int build_tables(sve_batch* b, int tile, int schedule) {
  const int n = b->nruns;
  std::vector<BatchRun<T>> runs(n);
  std::vector<int> order(n);
  for (int r = 0; r < n; ++r) order[r] = r;
  // largest runs first: their tiles start early, small runs fill the tail
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return (long long)b->P[x].nx * b->P[x].ny > (long long)b->P[y].nx * b->P[y].ny;
  });
  int pif = 0, pcell = 0;
  for (int r = 0; r < n; ++r) {
    runs[r].P = b->P[r];
    runs[r].S = run_state<T>(b, r);
    runs[r].ntile_if = (int)tiles_of(b->P[r].nfx + b->P[r].nfy, tile);
    runs[r].ntile_cell = (int)tiles_of((long long)b->P[r].nx * b->P[r].ny, tile);
    runs[r].part_if = pif;
    runs[r].part_cell = pcell;
    pif += runs[r].ntile_if;
    pcell += runs[r].ntile_cell;
  }
  std::vector<int2> tif, tcell;
  tif.reserve(pif);
  tcell.reserve(pcell);
  if (schedule == 0) {
    for (int r : order) {
      for (int k = 0; k < runs[r].ntile_if; ++k) tif.push_back(make_int2(r, k));
      for (int k = 0; k < runs[r].ntile_cell; ++k) tcell.push_back(make_int2(r, k));
    }
  } else {
    int maxif = 0, maxc = 0;
    for (int r = 0; r < n; ++r) { maxif = std::max(maxif, runs[r].ntile_if); maxc = std::max(maxc, runs[r].ntile_cell); }
    for (int k = 0; k < maxif; ++k)
      for (int r : order)
        if (k < runs[r].ntile_if) tif.push_back(make_int2(r, k));
    for (int k = 0; k < maxc; ++k)
      for (int r : order)
        if (k < runs[r].ntile_cell) tcell.push_back(make_int2(r, k));
  }
  if (b->d_tiles_if) cudaFree(b->d_tiles_if);
  if (b->d_tiles_cell) cudaFree(b->d_tiles_cell);
  b->d_tiles_if = nullptr;
  b->d_tiles_cell = nullptr;
  if (cudaMalloc(&b->d_tiles_if, sizeof(int2) * tif.size()) != cudaSuccess) return SVE_ERR_OOM;
  if (cudaMalloc(&b->d_tiles_cell, sizeof(int2) * tcell.size()) != cudaSuccess) return SVE_ERR_OOM;
  if (cudaMemcpy(b->d_tiles_if, tif.data(), sizeof(int2) * tif.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return SVE_ERR_CUDA;
  if (cudaMemcpy(b->d_tiles_cell, tcell.data(), sizeof(int2) * tcell.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return SVE_ERR_CUDA;
  if (cudaMemcpy(b->d_runs, runs.data(), sizeof(BatchRun<T>) * n, cudaMemcpyHostToDevice) != cudaSuccess)
    return SVE_ERR_CUDA;
  b->nt_if = (int)tif.size();
  b->nt_cell = (int)tcell.size();
  b->tile = tile;
  b->schedule = schedule;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  return SVE_OK;
}

int build_tables_any(sve_batch* b, int tile, int schedule) {
  return b->precision == SVE_FP64 ? build_tables<double>(b, tile, schedule) : build_tables<float>(b, tile, schedule);
}

template <typename T>
void launch_batch_step(sve_batch* b, cudaStream_t st) {
  const BatchRun<T>* runs = (const BatchRun<T>*)b->d_runs;
  if (b->tile == 128) {
    batch_interface_kernel<T, 128><<<b->nt_if, 128, 0, st>>>(runs, b->d_tiles_if, b->d_sc, b->d_spart);
    batch_cell_kernel<T, 128><<<b->nt_cell, 128, 0, st>>>(runs, b->d_tiles_cell, b->d_sc, b->d_mpart);
  } else {
    batch_interface_kernel<T, 256><<<b->nt_if, 256, 0, st>>>(runs, b->d_tiles_if, b->d_sc, b->d_spart);
    batch_cell_kernel<T, 256><<<b->nt_cell, 256, 0, st>>>(runs, b->d_tiles_cell, b->d_sc, b->d_mpart);
  }
}

void launch_batch_step_any(sve_batch* b, cudaStream_t st) {
  if (b->precision == SVE_FP64) launch_batch_step<double>(b, st);
  else launch_batch_step<float>(b, st);
}

int enqueue_batch(sve_batch* b, int nsteps) {
  for (int r = 0; r < b->nruns; ++r)
    if (!b->has_state[r]) return SVE_ERR_STATE;
  int done = 0;
  if (nsteps >= kBatchGraphSteps) {
    if (!b->graph) {
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SVE_ERR_CUDA;
      for (int s = 0; s < kBatchGraphSteps; ++s) launch_batch_step_any(b, b->capture);
      if (cudaStreamEndCapture(b->capture, &g) != cudaSuccess) return SVE_ERR_CUDA;
      const cudaError_t e = cudaGraphInstantiate(&b->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) { b->graph = nullptr; return SVE_ERR_CUDA; }
    }
    for (; done + kBatchGraphSteps <= nsteps; done += kBatchGraphSteps)
      if (cudaGraphLaunch(b->graph, b->stream) != cudaSuccess) return SVE_ERR_CUDA;
  }
  for (; done < nsteps; ++done) launch_batch_step_any(b, b->stream);
  if (cudaGetLastError() != cudaSuccess) return SVE_ERR_CUDA;
  b->last_launches = 2LL * nsteps;
  return SVE_OK;
}

int batch_status(sve_batch* b, std::vector<DevScalars>* out = nullptr) {
  std::vector<DevScalars> s(b->nruns);
  if (cudaMemcpyAsync(s.data(), b->d_sc, sizeof(DevScalars) * b->nruns, cudaMemcpyDeviceToHost, b->stream) !=
      cudaSuccess)
    return SVE_ERR_CUDA;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return SVE_ERR_CUDA;
  int st = 0;
  for (auto& x : s) st |= x.status;
  if (out) *out = s;
  if (st & sve::ST_NAN) return SVE_ERR_NAN;
  if (st & sve::ST_NEG_DEPTH) return SVE_ERR_NEG_DEPTH;
  if (st & sve::ST_RIEMANN) return SVE_ERR_RIEMANN;
  if (st & sve::ST_DT) return SVE_ERR_DT;
  return SVE_OK;
}

}  // namespace

extern "C" {

int sve_batch_create(const sve_config* cfgs, int nruns, sve_batch** out) {
  if (!cfgs || nruns < 1 || !out) return SVE_ERR_ARG;
  *out = nullptr;
  for (int r = 0; r < nruns; ++r) {
    const int rc = sve_internal_validate(&cfgs[r]);
    if (rc) return rc;
    if (cfgs[r].precision != cfgs[0].precision) return SVE_ERR_ARG;
  }
  sve_batch* b = new sve_batch();
  b->nruns = nruns;
  b->precision = cfgs[0].precision;
  b->elem = b->precision == SVE_FP64 ? 8 : 4;
  b->P.resize(nruns);
  b->off.resize(nruns);
  b->has_state.assign(nruns, 0);
  size_t bytes = 0;
  long long part_if = 0, part_cell = 0;
  for (int r = 0; r < nruns; ++r) {
    sve_internal_make_params(&cfgs[r], &b->P[r]);
    b->off[r] = bytes;
    bytes += run_bytes(b->P[r], b->elem);
    part_if += tiles_of(b->P[r].nfx + b->P[r].nfy, kTileSizes[0]);
    part_cell += tiles_of((long long)b->P[r].nx * b->P[r].ny, kTileSizes[0]);
  }
  b->arena_bytes = bytes;
  bool ok = cudaMalloc(&b->arena, bytes) == cudaSuccess;
  const size_t rec = b->precision == SVE_FP64 ? sizeof(BatchRun<double>) : sizeof(BatchRun<float>);
  ok = ok && cudaMalloc(&b->d_runs, rec * nruns) == cudaSuccess;
  ok = ok && cudaMalloc(&b->d_sc, sizeof(DevScalars) * nruns) == cudaSuccess;
  ok = ok && cudaMalloc(&b->d_spart, 2 * sizeof(double) * (size_t)part_if) == cudaSuccess;
  ok = ok && cudaMalloc(&b->d_mpart, 2 * sizeof(double) * (size_t)part_cell) == cudaSuccess;
  ok = ok && cudaMalloc(&b->d_init_part, 2 * sizeof(double) * (size_t)part_cell) == cudaSuccess;
  if (!ok) { sve_batch_destroy(b); return SVE_ERR_OOM; }
  if (cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) != cudaSuccess) { sve_batch_destroy(b); return SVE_ERR_CUDA; }
  cudaMemset(b->arena, 0, bytes);
  cudaMemset(b->d_sc, 0, sizeof(DevScalars) * nruns);
  const int rc = build_tables_any(b, 256, 0);
  if (rc || cudaDeviceSynchronize() != cudaSuccess) { sve_batch_destroy(b); return rc ? rc : SVE_ERR_CUDA; }
  *out = b;
  return SVE_OK;
}

int sve_batch_set_stream(sve_batch* b, void* stream) {
  if (!b) return SVE_ERR_ARG;
  b->stream = (cudaStream_t)stream;
  return SVE_OK;
}

int sve_batch_set_state(sve_batch* b, int run, const void* depth, const void* hu, const void* hv, const void* zb,
                        int where) {
  if (!b || run < 0 || run >= b->nruns || !depth || !hu || !zb) return SVE_ERR_ARG;
  if (where != SVE_HOST && where != SVE_DEVICE) return SVE_ERR_ARG;
  const DevParams& P = b->P[run];
  if (P.dim == 2 && !hv) return SVE_ERR_ARG;
  const size_t row = b->elem * (size_t)P.nx, pitch = b->elem * (size_t)P.ex;
  const size_t next = (size_t)(P.nx + 2) * (size_t)(P.ny + 2);
  const cudaMemcpyKind kind = where == SVE_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const void* src[4] = {depth, hu, P.dim == 2 ? hv : nullptr, zb};
  char* fields[4];
  if (b->precision == SVE_FP64) {
    DevState<double> S = run_state<double>(b, run);
    fields[0] = (char*)S.h; fields[1] = (char*)S.hu; fields[2] = (char*)S.hv; fields[3] = (char*)S.z;
  } else {
    DevState<float> S = run_state<float>(b, run);
    fields[0] = (char*)S.h; fields[1] = (char*)S.hu; fields[2] = (char*)S.hv; fields[3] = (char*)S.z;
  }
  for (int f = 0; f < 4; ++f) {
    if (src[f]) {
      if (cudaMemcpy2DAsync(fields[f] + b->elem * (size_t)(P.ex + 1), pitch, src[f], row, row, P.ny, kind,
                            b->stream) != cudaSuccess)
        return SVE_ERR_CUDA;
    } else if (cudaMemsetAsync(fields[f], 0, b->elem * next, b->stream) != cudaSuccess) {
      return SVE_ERR_CUDA;
    }
  }
  if (cudaMemsetAsync(b->d_sc + run, 0, sizeof(DevScalars), b->stream) != cudaSuccess) return SVE_ERR_CUDA;
  const int nb = (int)(((long long)P.nx * P.ny + sve::kThreads - 1) / sve::kThreads);
  if (b->precision == SVE_FP64)
    sve::init_kernel<double><<<nb, sve::kThreads, 0, b->stream>>>(P, run_state<double>(b, run), b->d_sc + run,
                                                                 b->d_init_part);
  else
    sve::init_kernel<float><<<nb, sve::kThreads, 0, b->stream>>>(P, run_state<float>(b, run), b->d_sc + run,
                                                                b->d_init_part);
  if (cudaGetLastError() != cudaSuccess) return SVE_ERR_CUDA;
  DevScalars s;
  if (cudaMemcpyAsync(&s, b->d_sc + run, sizeof(s), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
    return SVE_ERR_CUDA;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return SVE_ERR_CUDA;
  b->has_state[run] = 1;
  if (s.status & sve::ST_NAN) return SVE_ERR_NAN;
  if (s.status & sve::ST_NEG_DEPTH) return SVE_ERR_NEG_DEPTH;
  return SVE_OK;
}

int sve_batch_step(sve_batch* b, int nsteps) {
  if (!b || nsteps < 0) return SVE_ERR_ARG;
  const int rc = enqueue_batch(b, nsteps);
  if (rc) return rc;
  return batch_status(b);
}

int sve_batch_step_async(sve_batch* b, int nsteps) {
  if (!b || nsteps < 0) return SVE_ERR_ARG;
  return enqueue_batch(b, nsteps);
}

int sve_batch_get_state(sve_batch* b, int run, void* depth, void* hu, void* hv, void* zb, int where) {
  if (!b || run < 0 || run >= b->nruns) return SVE_ERR_ARG;
  if (!b->has_state[run]) return SVE_ERR_STATE;
  if (where != SVE_HOST && where != SVE_DEVICE) return SVE_ERR_ARG;
  const DevParams& P = b->P[run];
  const size_t row = b->elem * (size_t)P.nx, pitch = b->elem * (size_t)P.ex;
  const cudaMemcpyKind kind = where == SVE_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  char* fields[4];
  if (b->precision == SVE_FP64) {
    DevState<double> S = run_state<double>(b, run);
    fields[0] = (char*)S.h; fields[1] = (char*)S.hu; fields[2] = (char*)S.hv; fields[3] = (char*)S.z;
  } else {
    DevState<float> S = run_state<float>(b, run);
    fields[0] = (char*)S.h; fields[1] = (char*)S.hu; fields[2] = (char*)S.hv; fields[3] = (char*)S.z;
  }
  void* dst[4] = {depth, hu, hv, zb};
  for (int f = 0; f < 4; ++f) {
    if (!dst[f] || (f == 2 && P.dim == 1)) continue;
    if (cudaMemcpy2DAsync(dst[f], row, fields[f] + b->elem * (size_t)(P.ex + 1), pitch, row, P.ny, kind,
                          b->stream) != cudaSuccess)
      return SVE_ERR_CUDA;
  }
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return SVE_ERR_CUDA;
  return SVE_OK;
}

int sve_batch_get_diag(sve_batch* b, int run, double* mass_h, double* mass_z, double* t, double* last_dt) {
  if (!b || run < 0 || run >= b->nruns) return SVE_ERR_ARG;
  std::vector<DevScalars> s;
  const int rc = batch_status(b, &s);
  if (rc == SVE_ERR_CUDA) return rc;
  if (mass_h) *mass_h = s[run].mass_h;
  if (mass_z) *mass_z = s[run].mass_z;
  if (t) *t = s[run].t;
  if (last_dt) *last_dt = s[run].dt;
  return rc;
}

int sve_batch_get_counters(sve_batch* b, long long* steps, unsigned long long* newton_iters) {
  if (!b) return SVE_ERR_ARG;
  std::vector<DevScalars> s;
  const int rc = batch_status(b, &s);
  if (rc == SVE_ERR_CUDA) return rc;
  long long st = 0;
  unsigned long long it = 0;
  for (auto& x : s) { st += x.steps; it += x.newton_iters; }
  if (steps) *steps = st;
  if (newton_iters) *newton_iters = it;
  return rc;
}

int sve_batch_autotune(sve_batch* b, int trial_steps, int* tile, int* schedule) {
  if (!b || trial_steps < 1) return SVE_ERR_ARG;
  for (int r = 0; r < b->nruns; ++r)
    if (!b->has_state[r]) return SVE_ERR_STATE;
  // trials advance the runs: keep the state and scalars and restore them
  void* save = nullptr;
  std::vector<DevScalars> sc0(b->nruns);
  if (cudaMalloc(&save, b->arena_bytes) != cudaSuccess) return SVE_ERR_OOM;
  int rc = SVE_OK;
  if (cudaMemcpyAsync(save, b->arena, b->arena_bytes, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess ||
      cudaMemcpyAsync(sc0.data(), b->d_sc, sizeof(DevScalars) * b->nruns, cudaMemcpyDeviceToHost, b->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    rc = SVE_ERR_CUDA;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int best_tile = b->tile, best_sched = b->schedule;
  for (int ti = 0; ti < 2 && !rc; ++ti)
    for (int sc = 0; sc < kSchedules && !rc; ++sc) {
      rc = build_tables_any(b, kTileSizes[ti], sc);
      if (rc) break;
      launch_batch_step_any(b, b->stream);  // warm-up
      cudaEventRecord(e0, b->stream);
      for (int s = 0; s < trial_steps; ++s) launch_batch_step_any(b, b->stream);
      cudaEventRecord(e1, b->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) { rc = SVE_ERR_CUDA; break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) { best = ms; best_tile = kTileSizes[ti]; best_sched = sc; }
      // back to the saved state for the next candidate
      if (cudaMemcpyAsync(b->arena, save, b->arena_bytes, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess ||
          cudaMemcpyAsync(b->d_sc, sc0.data(), sizeof(DevScalars) * b->nruns, cudaMemcpyHostToDevice,
                          b->stream) != cudaSuccess ||
          cudaStreamSynchronize(b->stream) != cudaSuccess)
        rc = SVE_ERR_CUDA;
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(save);
  if (!rc) rc = build_tables_any(b, best_tile, best_sched);
  if (tile) *tile = best_tile;
  if (schedule) *schedule = best_sched;
  return rc;
}

int sve_batch_set_schedule(sve_batch* b, int tile, int schedule) {
  if (!b || (tile != 128 && tile != 256) || schedule < 0 || schedule >= kSchedules) return SVE_ERR_ARG;
  return build_tables_any(b, tile, schedule);
}

long long sve_batch_last_launch_count(sve_batch* b) { return b ? b->last_launches : -1; }

void sve_batch_destroy(sve_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->arena) cudaFree(b->arena);
  if (b->d_runs) cudaFree(b->d_runs);
  if (b->d_tiles_if) cudaFree(b->d_tiles_if);
  if (b->d_tiles_cell) cudaFree(b->d_tiles_cell);
  if (b->d_sc) cudaFree(b->d_sc);
  if (b->d_spart) cudaFree(b->d_spart);
  if (b->d_mpart) cudaFree(b->d_mpart);
  if (b->d_init_part) cudaFree(b->d_init_part);
  if (b->capture) cudaStreamDestroy(b->capture);
  delete b;
}

}  // extern "C"
