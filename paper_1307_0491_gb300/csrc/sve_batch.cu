// sve_batch.cu -- many independent runs of the step in one pair of launches
// per step (include/sve.h, sve_batch_*).
//
// Every run keeps its own grid, parameters, CFL time step, time and mass
// sums.  Work is cut into tiles of NT interfaces (or cells) of one run; a
// tile table lists the tiles of all runs in a schedule order, and each
// launch covers the whole table, so runs of uneven size share the GPU
// without one launch per run.  Each run's last tile to finish (an atomic
// ticket per run, no waiting) turns that run's running speed maxima into its
// time step (interface launch) or advances its time (cell launch); mass
// sums are reduced from per-tile partials when they are read.  The
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
#include "sve_fused.cuh"
#include "sve_march.cuh"

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
  int strips, rows, mtasks;  // FP32 2D (fused): strips, rows a run, strip-runs of this run
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
__global__ void __launch_bounds__(NT, sve::iface_min_blocks<NT>::value)
    batch_interface_kernel(const BatchRun<T>* runs, const int2* tiles, DevScalars* sc) {
  __shared__ BatchRun<T> R;
  // block tallies: maximal x / y speed (bit patterns), Newton updates, warps done
  __shared__ unsigned long long s_bits[2];
  __shared__ unsigned int s_its, s_warps, s_halv, s_raised, s_retry;
  const int2 t = tiles[blockIdx.x];
  if (threadIdx.x == 0) { s_bits[0] = 0ull; s_bits[1] = 0ull; s_its = 0u; s_warps = 0u; s_halv = 0u; s_raised = 0u; s_retry = 0u; }
  load_run(runs, t.x, &R);  // ends with a barrier
  const DevParams& P = R.P;
  const long long item = (long long)t.y * NT + threadIdx.x;
  double sx = 0.0, sy = 0.0;
  int iters = 0, branch = 0;
  bool fail = false;
  if (item < P.nfx) {
    fail = !sve::interface_item(P, R.S, false, item, sx, iters, branch);
  } else if (item < P.nfx + P.nfy) {
    fail = !sve::interface_item(P, R.S, true, item - P.nfx, sy, iters, branch);
  }
  if (fail) atomicOr(&sc[t.x].status, sve::ST_RIEMANN);
  // as in interface_kernel: warp shuffles, shared-memory atomics, no block
  // barrier; the block's last warp folds the tallies into the run's running
  // maxima (atomic max on the bit patterns: order-free), the run's last tile
  // turns them into its time step
  long long bx = __double_as_longlong(sx), by = __double_as_longlong(sy);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long ox = __shfl_xor_sync(0xffffffffu, bx, o), oy = __shfl_xor_sync(0xffffffffu, by, o);
    bx = ox > bx ? ox : bx;
    by = oy > by ? oy : by;
    iters += __shfl_xor_sync(0xffffffffu, iters, o);
  }
  const unsigned wb = __reduce_or_sync(0xffffffffu, (unsigned)branch);
  unsigned wr = 0u, wt = 0u, wh = 0u;
  if (wb) {
    wr = __reduce_add_sync(0xffffffffu, sve::branch_raised(branch));
    wt = __reduce_add_sync(0xffffffffu, sve::branch_retries(branch));
    wh = __reduce_add_sync(0xffffffffu, sve::branch_halvings(branch));
  }
  if ((threadIdx.x & 31) != 0) return;
  atomicMax(&s_bits[0], (unsigned long long)bx);
  atomicMax(&s_bits[1], (unsigned long long)by);
  atomicAdd(&s_its, (unsigned int)iters);
  if (wb) { atomicAdd(&s_raised, wr); atomicAdd(&s_retry, wt); atomicAdd(&s_halv, wh); }
  __threadfence_block();
  if (atomicAdd(&s_warps, 1u) != NT / 32 - 1) return;
  __threadfence_block();
  DevScalars& S = sc[t.x];
  atomicAdd(&S.newton_iters, (unsigned long long)atomicAdd(&s_its, 0u));
  const unsigned br = atomicAdd(&s_raised, 0u), bt = atomicAdd(&s_retry, 0u), bh = atomicAdd(&s_halv, 0u);
  if (bt) atomicAdd(&S.retries, (unsigned long long)bt);
  if (br) atomicAdd(&S.raised, (unsigned long long)br);
  if (bh) atomicAdd(&S.halvings, (unsigned long long)bh);
  atomicMax(&S.smax_bits[0], atomicMax(&s_bits[0], 0ull));
  atomicMax(&S.smax_bits[1], atomicMax(&s_bits[1], 0ull));
  __threadfence();
  if (atomicAdd(&S.done_iface, 1u) != (unsigned)R.ntile_if - 1) return;
  __threadfence();
  const double mx = __longlong_as_double((long long)atomicExch(&S.smax_bits[0], 0ull));
  const double my = __longlong_as_double((long long)atomicExch(&S.smax_bits[1], 0ull));
  double dt = (P.dim == 1) ? P.cfl * P.dx / mx : P.cfl / (mx / P.dx + my / P.dy);
  if (!(dt > 0.0) || !isfinite(dt)) { atomicOr(&S.status, sve::ST_DT); dt = 0.0; }
  S.dt = dt;
  S.Sx = mx;
  S.Sy = my;
  S.done_iface = 0u;
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT) batch_cell_kernel(const BatchRun<T>* runs, const int2* tiles, DevScalars* sc,
                                                        double* mpart) {
  __shared__ BatchRun<T> R;
  __shared__ double s_m[2][NT];
  __shared__ unsigned int s_warps;
  const int2 t = tiles[blockIdx.x];
  if (threadIdx.x == 0) s_warps = 0u;
  load_run(runs, t.x, &R);  // ends with a barrier
  const DevParams& P = R.P;
  const long long k = (long long)t.y * NT + threadIdx.x;
  double mh = 0.0, mz = 0.0;
  if (k < (long long)P.nx * P.ny) {
    const int st = sve::cell_item(P, R.S, k, sc[t.x].dt, mh, mz);
    if (st) atomicOr(&sc[t.x].status, st);
  }
  // the tile's mass partial in a fixed order by the block's last warp (as in
  // cell_kernel); the run's sums are reduced from the partials on read-out
  s_m[0][threadIdx.x] = mh;
  s_m[1][threadIdx.x] = mz;
  __syncwarp();
  unsigned int w = 0u;
  if ((threadIdx.x & 31) == 0) {
    __threadfence_block();
    w = atomicAdd(&s_warps, 1u);
  }
  w = __shfl_sync(0xffffffffu, w, 0);
  if (w != NT / 32 - 1) return;
  __threadfence_block();
  const int lane = threadIdx.x & 31;
  double a = 0.0, b = 0.0;
#pragma unroll
  for (int q = 0; q < NT / 32; ++q) { a += s_m[0][lane + 32 * q]; b += s_m[1][lane + 32 * q]; }
  a = sve::warp_sum(a);
  b = sve::warp_sum(b);
  if (lane != 0) return;
  mpart[2 * (R.part_cell + t.y)] = a;
  mpart[2 * (R.part_cell + t.y) + 1] = b;
  __threadfence();
  DevScalars& S = sc[t.x];
  if (atomicAdd(&S.done_cell, 1u) != (unsigned)R.ntile_cell - 1) return;
  S.mass_parts = (unsigned)R.ntile_cell;
  S.t += S.dt;
  S.steps += 1;
  S.done_cell = 0u;
}

// FP32 2D runs: the solve pass as column strips marching over rows
// (march_task of sve_march.cuh), four strip-runs of one run per block; the
// run's last block turns its speed maxima into its time step.  Four blocks
// per SM: the run record in shared memory costs registers that five blocks
// (<= 102) would spill.
// The two state buffers of a run for the carried update (p = 0: its state;
// 1: its projection planes tau, u, v, pi, which the FP32 2D form does not
// use) and the two halves of its fluctuation planes.
template <typename T>
__device__ __forceinline__ sve::StateBuf<T> run_buf(const BatchRun<T>& R, int p) {
  if (p) return {R.S.tau, R.S.u, R.S.v, R.S.pi};
  return {R.S.h, R.S.hu, R.S.hv, R.S.z};
}
template <typename T>
__device__ __forceinline__ sve::NetFluct<T> run_dF(const BatchRun<T>& R, int p) {
  const long long ncell = (long long)R.P.nx * R.P.ny;
  T* b = R.S.fx + (long long)p * 4 * ncell;  // 8 (nx + 1) ny >= 8 nx ny
  return {b, b + ncell, b + 2 * ncell, b + 3 * ncell};
}

// carry < 0: a plain solve pass on the runs' states; carry = q >= 0: the
// carried form of a call's step k >= 1 with q = (k - 1) % 2 (as the single
// run's: U^{k-1} in buffer q, the update of step k - 1 in half q, U^k to
// buffer 1 - q, this step's net fluctuations to half 1 - q).
template <typename T>
__global__ void __launch_bounds__(sve::kMThreads, 4) batch_march_kernel(const BatchRun<T>* runs, const int2* tiles,
                                                                        DevScalars* sc, int carry) {
  __shared__ BatchRun<T> R;
  __shared__ unsigned long long s_sx, s_sy;
  __shared__ unsigned int s_cnt[5];
  const int2 t = tiles[blockIdx.x];
  if (threadIdx.x == 0) { s_sx = 0ull; s_sy = 0ull; for (int k = 0; k < 5; ++k) s_cnt[k] = 0u; }
  load_run(runs, t.x, &R);  // ends with a barrier
  const DevParams& P = R.P;
  const int task = t.y * sve::kMWarps + (int)(threadIdx.x >> 5);
  sve::MarchTally<T> tl;
  if (task < R.mtasks) {
    const int q = carry < 0 ? 0 : carry;
    const sve::Carry<T> K{run_buf(R, 1 - q), run_dF(R, q), carry < 0 ? T(0) : T(sc[t.x].dt)};
    sve::march_task(P, run_buf(R, q), run_dF(R, carry < 0 ? 0 : 1 - q), task % R.strips, task / R.strips, R.rows,
                    tl, carry >= 0, K);
  }
  DevScalars& S = sc[t.x];
  if (!sve::march_fold(tl, &S, &s_sx, &s_sy, s_cnt)) return;
  __threadfence();
  if (atomicAdd(&S.done_iface, 1u) != (unsigned)R.ntile_if - 1) return;
  __threadfence();
  const double mx = __longlong_as_double((long long)atomicExch(&S.smax_bits[0], 0ull));
  const double my = __longlong_as_double((long long)atomicExch(&S.smax_bits[1], 0ull));
  if (carry >= 0) {  // the carried step is complete (its mass sums: from the final apply pass)
    S.t += S.dt;
    S.steps += 1;
  }
  double dt = P.cfl / (mx / P.dx + my / P.dy);
  if (!(dt > 0.0) || !isfinite(dt)) { atomicOr(&S.status, sve::ST_DT); dt = 0.0; }
  S.dt = dt;
  S.Sx = mx;
  S.Sy = my;
  S.done_iface = 0u;
}

// FP32 2D runs: the update from the net fluctuations (apply_cell of
// sve_fused.cuh), one cell a thread over tiles of NT cells of one run.
// q: the buffer and half holding the state and update the pass applies
// (the new state goes to buffer 0).
template <typename T, int NT>
__global__ void __launch_bounds__(NT) batch_apply_kernel(const BatchRun<T>* runs, const int2* tiles, DevScalars* sc,
                                                         double* mpart, int q) {
  __shared__ BatchRun<T> R;
  __shared__ double s_m[2][NT];
  __shared__ unsigned int s_warps;
  const int2 t = tiles[blockIdx.x];
  if (threadIdx.x == 0) s_warps = 0u;
  load_run(runs, t.x, &R);  // ends with a barrier
  const DevParams& P = R.P;
  const long long k = (long long)t.y * NT + threadIdx.x;
  double mh = 0.0, mz = 0.0;
  if (k < (long long)P.nx * P.ny) {
    const int j = (int)(k / P.nx), i = (int)(k - (long long)j * P.nx);
    T h1, z1;
    const int st =
        sve::apply_cell(P, run_buf(R, q), run_buf(R, 0), run_dF(R, q), T(sc[t.x].dt), i, j, sve::Mirror<T>{}, h1, z1);
    if (st) atomicOr(&sc[t.x].status, st);
    mh = (double)h1;
    mz = (double)z1;
  }
  s_m[0][threadIdx.x] = mh;
  s_m[1][threadIdx.x] = mz;
  __syncwarp();
  unsigned int w = 0u;
  if ((threadIdx.x & 31) == 0) {
    __threadfence_block();
    w = atomicAdd(&s_warps, 1u);
  }
  w = __shfl_sync(0xffffffffu, w, 0);
  if (w != NT / 32 - 1) return;
  __threadfence_block();
  const int lane = threadIdx.x & 31;
  double a = 0.0, b = 0.0;
#pragma unroll
  for (int q = 0; q < NT / 32; ++q) { a += s_m[0][lane + 32 * q]; b += s_m[1][lane + 32 * q]; }
  a = sve::warp_sum(a);
  b = sve::warp_sum(b);
  if (lane != 0) return;
  mpart[2 * (R.part_cell + t.y)] = a;
  mpart[2 * (R.part_cell + t.y) + 1] = b;
  __threadfence();
  DevScalars& S = sc[t.x];
  if (atomicAdd(&S.done_cell, 1u) != (unsigned)R.ntile_cell - 1) return;
  S.mass_parts = (unsigned)R.ntile_cell;
  S.t += S.dt;
  S.steps += 1;
  S.done_cell = 0u;
}

// Mass sums of one run from its per-tile (or, after an upload, per-block)
// partials, in a fixed order (one block; launched when they are read).
__global__ void __launch_bounds__(sve::kThreads) batch_mass_kernel(const double* part, DevScalars* S, double cell) {
  __shared__ double sh[2 * (sve::kThreads / 32)];
  double a, b;
  sve::reduce_partials<sve::kThreads>(part, S->mass_parts, a, b, sh);
  if (threadIdx.x == 0) {
    S->mass_h = a * cell;
    S->mass_z = b * cell;
  }
}

constexpr int kBatchGraphSteps = 8;
constexpr int kTileSizes[2] = {128, 256};
constexpr int kSchedules = 2;  // 0: run after run (largest first), 1: round robin over runs
constexpr int kMarchRows[4] = {8, 16, 32, 64};  // rows a strip-run of the FP32 2D batch (autotuner's choices)

}  // namespace

__attribute__((visibility("hidden"))) int sve_internal_validate(const sve_config* c);
__attribute__((visibility("hidden"))) bool sve_internal_has_external(const sve_config* c);
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
  double* d_mpart = nullptr;
  double* d_init_part = nullptr;     // partials for the per-run init kernel
  std::vector<int> part_cell;        // first cell partial of each run at the current tile size
  // where a run's mass sums come from when read: 0 the upload's partials
  // (d_init_part, transient: reduced at once), 1 the last step's partials
  // (d_mpart), 2 the scalars themselves (already reduced)
  std::vector<int> mass_src;
  int tile = 128, schedule = 0;
  bool fused = false;                // FP32 state, every run 2D: the marching solve pass + apply pass
  int rows = 32;                     // rows a strip-run of the fused solve pass
  struct Trial { int tile, schedule, rows; float ms_per_step; };
  std::vector<Trial> trials;         // the last autotune's candidates and their times
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
    runs[r].strips = (b->P[r].nx + sve::kMCols - 1) / sve::kMCols;
    runs[r].rows = b->rows;
    runs[r].mtasks = runs[r].strips * ((b->P[r].ny + b->rows - 1) / b->rows);
    runs[r].ntile_if = b->fused ? (int)tiles_of(runs[r].mtasks, sve::kMWarps)
                                : (int)tiles_of(b->P[r].nfx + b->P[r].nfy, tile);
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
  b->part_cell.resize(n);
  for (int r = 0; r < n; ++r) b->part_cell[r] = runs[r].part_cell;
  b->tile = tile;
  b->schedule = schedule;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  return SVE_OK;
}

int build_tables_any(sve_batch* b, int tile, int schedule) {
  return b->precision == SVE_FP64 ? build_tables<double>(b, tile, schedule) : build_tables<float>(b, tile, schedule);
}

// The fused FP32 2D passes: the solve pass (carry as batch_march_kernel's)
// and the apply pass from buffer q.
void launch_batch_march(sve_batch* b, cudaStream_t st, int carry) {
  batch_march_kernel<float><<<b->nt_if, sve::kMThreads, 0, st>>>((const BatchRun<float>*)b->d_runs, b->d_tiles_if,
                                                                 b->d_sc, carry);
}
void launch_batch_apply(sve_batch* b, cudaStream_t st, int q) {
  const BatchRun<float>* runs = (const BatchRun<float>*)b->d_runs;
  if (b->tile == 128)
    batch_apply_kernel<float, 128><<<b->nt_cell, 128, 0, st>>>(runs, b->d_tiles_cell, b->d_sc, b->d_mpart, q);
  else
    batch_apply_kernel<float, 256><<<b->nt_cell, 256, 0, st>>>(runs, b->d_tiles_cell, b->d_sc, b->d_mpart, q);
}

template <typename T>
void launch_batch_step(sve_batch* b, cudaStream_t st) {
  const BatchRun<T>* runs = (const BatchRun<T>*)b->d_runs;
  if (b->fused) {
    launch_batch_march(b, st, -1);
    launch_batch_apply(b, st, 0);
    return;
  }
  if (b->tile == 128) {
    batch_interface_kernel<T, 128><<<b->nt_if, 128, 0, st>>>(runs, b->d_tiles_if, b->d_sc);
    batch_cell_kernel<T, 128><<<b->nt_cell, 128, 0, st>>>(runs, b->d_tiles_cell, b->d_sc, b->d_mpart);
  } else {
    batch_interface_kernel<T, 256><<<b->nt_if, 256, 0, st>>>(runs, b->d_tiles_if, b->d_sc);
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
  if (b->fused && nsteps > 1) {
    // the carried update (as a single run's call): step 0, steps 1 .. n - 1
    // (graphs of kBatchGraphSteps carried solve passes from buffer 0), the
    // apply pass
    launch_batch_march(b, b->stream, -1);
    int k = 1;
    if (nsteps - 1 >= kBatchGraphSteps) {
      if (!b->graph) {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SVE_ERR_CUDA;
        for (int s = 0; s < kBatchGraphSteps; ++s) launch_batch_march(b, b->capture, s & 1);
        if (cudaStreamEndCapture(b->capture, &g) != cudaSuccess) return SVE_ERR_CUDA;
        const cudaError_t e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { b->graph = nullptr; return SVE_ERR_CUDA; }
      }
      for (; k + kBatchGraphSteps <= nsteps; k += kBatchGraphSteps)
        if (cudaGraphLaunch(b->graph, b->stream) != cudaSuccess) return SVE_ERR_CUDA;
    }
    for (; k < nsteps; ++k) launch_batch_march(b, b->stream, (k - 1) & 1);
    launch_batch_apply(b, b->stream, (nsteps - 1) & 1);
    if (cudaGetLastError() != cudaSuccess) return SVE_ERR_CUDA;
    std::fill(b->mass_src.begin(), b->mass_src.end(), 1);
    b->last_launches = (long long)nsteps + 1;
    return SVE_OK;
  }
  int done = 0;
  if (nsteps >= kBatchGraphSteps) {
    if (!b->graph) {
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SVE_ERR_CUDA;
      for (int s = 0; s < kBatchGraphSteps; ++s) launch_batch_step_any(b, b->capture);  // (not fused FP32 2D)
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
  if (nsteps > 0) std::fill(b->mass_src.begin(), b->mass_src.end(), 1);
  b->last_launches = 2LL * nsteps;
  return SVE_OK;
}

// Reduce run r's mass sums into its scalars from where they currently are.
int reduce_mass(sve_batch* b, int r) {
  if (!b->has_state[r] || b->mass_src[r] == 2) return SVE_OK;
  const DevParams& P = b->P[r];
  const double* part = b->mass_src[r] == 1 ? b->d_mpart + 2 * (size_t)b->part_cell[r] : b->d_init_part;
  batch_mass_kernel<<<1, sve::kThreads, 0, b->stream>>>(part, b->d_sc + r, P.dx * (P.dim == 2 ? P.dy : 1.0));
  return cudaGetLastError() == cudaSuccess ? SVE_OK : SVE_ERR_CUDA;
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
    int rc = sve_internal_validate(&cfgs[r]);
    if (!rc && sve_internal_has_external(&cfgs[r])) rc = SVE_ERR_ARG;  // no block calls on a batch
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
  b->mass_src.assign(nruns, 0);
  size_t bytes = 0;
  long long part_cell = 0;
  for (int r = 0; r < nruns; ++r) {
    sve_internal_make_params(&cfgs[r], &b->P[r]);
    b->off[r] = bytes;
    bytes += run_bytes(b->P[r], b->elem);
    part_cell += tiles_of((long long)b->P[r].nx * b->P[r].ny, kTileSizes[0]);
  }
  b->arena_bytes = bytes;
  b->fused = b->precision == SVE_FP32;
  for (int r = 0; r < nruns; ++r) b->fused = b->fused && cfgs[r].dim == 2;
  bool ok = cudaMalloc(&b->arena, bytes) == cudaSuccess;
  const size_t rec = b->precision == SVE_FP64 ? sizeof(BatchRun<double>) : sizeof(BatchRun<float>);
  ok = ok && cudaMalloc(&b->d_runs, rec * nruns) == cudaSuccess;
  ok = ok && cudaMalloc(&b->d_sc, sizeof(DevScalars) * nruns) == cudaSuccess;
  ok = ok && cudaMalloc(&b->d_mpart, 2 * sizeof(double) * (size_t)part_cell) == cudaSuccess;
  ok = ok && cudaMalloc(&b->d_init_part, 2 * sizeof(double) * (size_t)part_cell) == cudaSuccess;
  if (!ok) { sve_batch_destroy(b); return SVE_ERR_OOM; }
  if (cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) != cudaSuccess) { sve_batch_destroy(b); return SVE_ERR_CUDA; }
  cudaMemset(b->arena, 0, bytes);
  cudaMemset(b->d_sc, 0, sizeof(DevScalars) * nruns);
  const int rc = build_tables_any(b, 128, 0);
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
  // the upload's mass sums now: the init partials buffer is shared by the runs
  b->has_state[run] = 1;
  b->mass_src[run] = 0;
  if (reduce_mass(b, run)) return SVE_ERR_CUDA;
  b->mass_src[run] = 2;
  DevScalars s;
  if (cudaMemcpyAsync(&s, b->d_sc + run, sizeof(s), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
    return SVE_ERR_CUDA;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return SVE_ERR_CUDA;
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
  if (reduce_mass(b, run)) return SVE_ERR_CUDA;
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
  // trials advance the runs: keep the state and scalars (with the mass sums
  // reduced first, since the trials overwrite the partials) and restore them
  for (int r = 0; r < b->nruns; ++r) {
    if (reduce_mass(b, r)) return SVE_ERR_CUDA;
    b->mass_src[r] = 2;
  }
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
  int best_tile = b->tile, best_sched = b->schedule, best_rows = b->rows;
  b->trials.clear();
  // candidates: the tile size of the per-item launches (the cell or apply
  // pass, and the interface pass of the two-kernel form), the tile order,
  // and for the fused FP32 2D form the rows of a strip-run (the solve
  // pass's tile: 30 columns x rows)
  const int nrows = b->fused ? 4 : 1;
  for (int ri = 0; ri < nrows && !rc; ++ri)
    for (int ti = 0; ti < 2 && !rc; ++ti)
      for (int sc = 0; sc < kSchedules && !rc; ++sc) {
        if (b->fused) b->rows = kMarchRows[ri];
        rc = build_tables_any(b, kTileSizes[ti], sc);
        if (rc) break;
        launch_batch_step_any(b, b->stream);  // warm-up
        cudaEventRecord(e0, b->stream);
        for (int s = 0; s < trial_steps; ++s) launch_batch_step_any(b, b->stream);
        cudaEventRecord(e1, b->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = SVE_ERR_CUDA; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        b->trials.push_back({kTileSizes[ti], sc, b->fused ? b->rows : 0, ms / (float)trial_steps});
        if (ms < best) { best = ms; best_tile = kTileSizes[ti]; best_sched = sc; best_rows = b->rows; }
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
  b->rows = best_rows;
  if (!rc) rc = build_tables_any(b, best_tile, best_sched);
  if (tile) *tile = best_tile;
  if (schedule) *schedule = best_sched;
  return rc;
}

int sve_batch_autotune_trials(sve_batch* b, int n, int* tile, int* schedule, int* rows, double* ms_per_step) {
  if (!b || n < 0) return SVE_ERR_ARG;
  const int m = std::min(n, (int)b->trials.size());
  for (int k = 0; k < m; ++k) {
    if (tile) tile[k] = b->trials[k].tile;
    if (schedule) schedule[k] = b->trials[k].schedule;
    if (rows) rows[k] = b->trials[k].rows;
    if (ms_per_step) ms_per_step[k] = b->trials[k].ms_per_step;
  }
  return (int)b->trials.size();
}

int sve_batch_set_rows(sve_batch* b, int rows) {
  if (!b || !b->fused || (rows != 8 && rows != 16 && rows != 32 && rows != 64)) return SVE_ERR_ARG;
  b->rows = rows;
  return build_tables_any(b, b->tile, b->schedule);
}

int sve_batch_get_rows(sve_batch* b) {
  if (!b) return SVE_ERR_ARG;
  return b->fused ? b->rows : 0;
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
  if (b->d_mpart) cudaFree(b->d_mpart);
  if (b->d_init_part) cudaFree(b->d_init_part);
  if (b->capture) cudaStreamDestroy(b->capture);
  delete b;
}

}  // extern "C"
