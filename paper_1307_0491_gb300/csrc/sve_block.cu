// sve_block.cu -- one block of a domain decomposition (Sec. 4 of
// arXiv:1307.0491: the grid is cut into blocks, each with one ghost layer
// that the neighbouring blocks fill before every step, and the time step is
// the minimum over all blocks of their CFL steps).
//
// A handle whose configuration marks a side SVE_BC_EXTERNAL steps one block:
// its own boundary rules fill the other sides, and the caller fills the
// external sides' ghost ring from the neighbours' edge cells
// (sve_block_get_edge on the neighbour, sve_block_set_ghosts here).  A step
// is split where the blocks have to agree on the time step:
// sve_block_speeds solves every interface of the block and returns its
// extreme wave speeds; the caller takes the maximum over all blocks and
// sve_block_advance updates the cells with the CFL step of that maximum.
// The kernels are the ones a whole-grid step runs, so a decomposed run
// equals the whole-grid run cell for cell (with the same launch shape of the
// two-kernel step: sve_set_block_size).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include "../../include/sve.h"
#include "sve_device.cuh"
#include "sve_fused.cuh"
#include "sve_handle.h"
#include "sve_march.cuh"

__attribute__((visibility("hidden"))) int sve_internal_status_code(int st);
__attribute__((visibility("hidden"))) int sve_internal_reserve_dtlog(sve_handle* h, int n);

namespace {

using sve::DevParams;
using sve::DevScalars;

// The ghost ring of one side from n cells (h, hu, hv, z planes of n values):
// stored and projected as the boundary rules' ghosts are; a non-finite value
// or a depth <= 0 is latched in the status word.
template <typename T>
__global__ void __launch_bounds__(sve::kThreads) ghost_set_kernel(DevParams P, sve::DevState<T> S, DevScalars* sc,
                                                                  int side, const T* in, int n) {
  const int k = blockIdx.x * sve::kThreads + threadIdx.x;
  if (k >= n) return;
  const int i = side == 0 ? -1 : (side == 1 ? P.nx : k);
  const int j = side < 2 ? k : (side == 2 ? -1 : P.ny);
  T s[4] = {in[k], in[n + k], P.dim == 2 ? in[2 * n + k] : T(0), in[3 * n + k]};
  if (!(sve::tfinite(s[0]) && sve::tfinite(s[1]) && sve::tfinite(s[2]) && sve::tfinite(s[3])))
    atomicOr(&sc->status, sve::ST_NAN);
  else if (!sve::positive(s[0]))
    atomicOr(&sc->status, sve::ST_NEG_DEPTH);
  sve::store_cell(P, S, sve::ext_index(P, i, j), s, sve::tdiv(T(1), s[0]));
}

bool side_ok(const sve_handle* h, int side) {
  return side >= 0 && side < (h->cfg.dim == 2 ? 4 : 2);
}

int side_len(const sve_handle* h, int side) { return side < 2 ? h->P.ny : h->P.nx; }

int wait_status(sve_handle* h, DevScalars* out = nullptr) {
  DevScalars s;
  if (cudaMemcpyAsync(&s, h->sc, sizeof(s), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess) return SVE_ERR_CUDA;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SVE_ERR_CUDA;
  h->last_t = s.t;
  if (out) *out = s;
  return sve_internal_status_code(s.status);
}

template <typename T>
void launch_solve(sve_handle* h) {
  const sve::DevState<T> S = state_of<T>(h);
  if (h->fused) {
    if constexpr (sizeof(T) == 4) {
      sve::StateBuf<T> B = {S.h, S.hu, S.hv, S.z};
      const size_t ncell = (size_t)h->P.nx * (size_t)h->P.ny;
      sve::NetFluct<T> D;
      D.h = (T*)h->fx; D.hu = D.h + ncell; D.hv = D.hu + ncell; D.z = D.hv + ncell;
      const sve::MarchShape& M = h->march;
      sve::march_kernel<T><<<M.blocks, sve::kMThreads, 0, h->stream>>>(h->P, B, D, h->sc, h->fixed, h->dtlog,
                                                                       sve::DT_SPEEDS_ONLY, M.strips, M.rows,
                                                                       M.tasks);
    }
    return;
  }
  const unsigned nbi = (unsigned)sve::iface_blocks(h->P, h->nt);
  if (h->nt == sve::kThreadsNarrow)
    sve::interface_kernel<T, sve::kThreadsNarrow><<<nbi, h->nt, 0, h->stream>>>(h->P, S, h->sc, h->fixed, h->dtlog,
                                                                                 sve::DT_SPEEDS_ONLY);
  else if (h->nt == sve::kThreadsStep)
    sve::interface_kernel<T, sve::kThreadsStep><<<nbi, h->nt, 0, h->stream>>>(h->P, S, h->sc, h->fixed, h->dtlog,
                                                                              sve::DT_SPEEDS_ONLY);
  else
    sve::interface_kernel<T, sve::kThreads><<<nbi, h->nt, 0, h->stream>>>(h->P, S, h->sc, h->fixed, h->dtlog,
                                                                          sve::DT_SPEEDS_ONLY);
}

template <typename T>
void launch_update(sve_handle* h) {
  const sve::DevState<T> S = state_of<T>(h);
  if (h->fused) {
    if constexpr (sizeof(T) == 4) {
      sve::StateBuf<T> B = {S.h, S.hu, S.hv, S.z};
      const size_t ncell = (size_t)h->P.nx * (size_t)h->P.ny;
      sve::NetFluct<T> D;
      D.h = (T*)h->fx; D.hu = D.h + ncell; D.hv = D.hu + ncell; D.z = D.hv + ncell;
      sve::apply_kernel<T><<<dim3(h->agx, h->agy), sve::kAThreads, 0, h->stream>>>(h->P, B, B, D, h->sc, h->mpart,
                                                                                     sve::Mirror<T>{});
    }
    return;
  }
  const unsigned nbc = (unsigned)sve::cell_blocks(h->P, h->nt);
  if (h->nt == sve::kThreadsNarrow)
    sve::cell_kernel<T, sve::kThreadsNarrow><<<nbc, h->nt, 0, h->stream>>>(h->P, S, h->sc, h->mpart, sve::Mirror<T>{});
  else if (h->nt == sve::kThreadsStep)
    sve::cell_kernel<T, sve::kThreadsStep><<<nbc, h->nt, 0, h->stream>>>(h->P, S, h->sc, h->mpart, sve::Mirror<T>{});
  else
    sve::cell_kernel<T, sve::kThreads><<<nbc, h->nt, 0, h->stream>>>(h->P, S, h->sc, h->mpart, sve::Mirror<T>{});
}

}  // namespace

extern "C" {

int sve_block_get_edge(sve_handle* h, int side, void* edge, int where) {
  if (!h || !edge || !side_ok(h, side) || (where != SVE_HOST && where != SVE_DEVICE)) return SVE_ERR_ARG;
  if (!h->has_state) return SVE_ERR_STATE;
  const DevParams& P = h->P;
  const int n = side_len(h, side);
  const size_t es = h->elem, pitch = es * (size_t)P.ex;
  const cudaMemcpyKind kind = where == SVE_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  // the interior cells along the side: column 0 / nx - 1, row 0 / ny - 1
  const int i = side == 0 ? 0 : (side == 1 ? P.nx - 1 : 0);
  const int j = side == 2 ? 0 : (side == 3 ? P.ny - 1 : 0);
  const size_t off = es * ((size_t)(j + 1) * (size_t)P.ex + (size_t)(i + 1));  // padded index of (i, j)
  for (int f = 0; f < 4; ++f) {
    char* dst = (char*)edge + es * (size_t)n * (size_t)f;
    if (f == 2 && P.dim == 1) {  // no hv in 1D: zeros
      if (where == SVE_HOST) memset(dst, 0, es * (size_t)n);
      else if (cudaMemsetAsync(dst, 0, es * (size_t)n, h->stream) != cudaSuccess) return SVE_ERR_CUDA;
      continue;
    }
    const char* src = (const char*)h->fields[f] + off;
    cudaError_t e = side < 2 ? cudaMemcpy2DAsync(dst, es, src, pitch, es, (size_t)n, kind, h->stream)
                             : cudaMemcpyAsync(dst, src, es * (size_t)n, kind, h->stream);
    if (e != cudaSuccess) return SVE_ERR_CUDA;
  }
  return cudaStreamSynchronize(h->stream) == cudaSuccess ? SVE_OK : SVE_ERR_CUDA;
}

int sve_block_set_ghosts(sve_handle* h, int side, const void* ghosts, int where) {
  if (!h || !ghosts || !side_ok(h, side) || (where != SVE_HOST && where != SVE_DEVICE)) return SVE_ERR_ARG;
  if (h->cfg.bc[side] != SVE_BC_EXTERNAL) return SVE_ERR_ARG;
  if (!h->has_state) return SVE_ERR_STATE;
  const DevParams& P = h->P;
  const size_t cap = 4 * h->elem * (size_t)(P.nx > P.ny ? P.nx : P.ny);
  if (!h->halo && cudaMalloc(&h->halo, cap) != cudaSuccess) return SVE_ERR_OOM;
  const int n = side_len(h, side);
  const size_t bytes = 4 * h->elem * (size_t)n;
  const void* src = ghosts;
  if (where == SVE_HOST) {
    if (cudaMemcpyAsync(h->halo, ghosts, bytes, cudaMemcpyHostToDevice, h->stream) != cudaSuccess) return SVE_ERR_CUDA;
    src = h->halo;
  }
  const unsigned nb = (unsigned)((n + sve::kThreads - 1) / sve::kThreads);
  if (h->cfg.precision == SVE_FP64)
    ghost_set_kernel<double><<<nb, sve::kThreads, 0, h->stream>>>(P, state_of<double>(h), h->sc, side,
                                                                  (const double*)src, n);
  else
    ghost_set_kernel<float><<<nb, sve::kThreads, 0, h->stream>>>(P, state_of<float>(h), h->sc, side,
                                                                 (const float*)src, n);
  if (cudaGetLastError() != cudaSuccess) return SVE_ERR_CUDA;
  // a host buffer may be reused by the caller as soon as this returns
  if (where == SVE_HOST && cudaStreamSynchronize(h->stream) != cudaSuccess) return SVE_ERR_CUDA;
  return SVE_OK;
}

int sve_block_speeds(sve_handle* h, double* sx, double* sy) {
  if (!h || !sx) return SVE_ERR_ARG;
  if (!h->has_state) return SVE_ERR_STATE;
  int rc = sve_internal_reserve_dtlog(h, 1);
  if (rc) return rc;
  if (cudaMemsetAsync(&h->sc->call_step, 0, sizeof(int), h->stream) != cudaSuccess) return SVE_ERR_CUDA;
  if (h->cfg.precision == SVE_FP64) launch_solve<double>(h);
  else launch_solve<float>(h);
  if (cudaGetLastError() != cudaSuccess) return SVE_ERR_CUDA;
  DevScalars s;
  rc = wait_status(h, &s);
  *sx = s.Sx;
  if (sy) *sy = h->cfg.dim == 2 ? s.Sy : 0.0;
  h->last_launches = 1;
  h->last_steps = 0;
  return rc;
}

int sve_block_advance(sve_handle* h, double sx, double sy) {
  if (!h) return SVE_ERR_ARG;
  if (!h->has_state) return SVE_ERR_STATE;
  const DevParams& P = h->P;
  // the CFL step of the maxima over all blocks, by the formula the solve
  // pass of a whole-grid step uses (reading R5)
  const double dt = P.dim == 1 ? P.cfl * P.dx / sx : P.cfl / (sx / P.dx + sy / P.dy);
  if (!(dt > 0.0) || !isfinite(dt)) return SVE_ERR_DT;
  int rc = sve_internal_reserve_dtlog(h, 1);
  if (rc) return rc;
  if (cudaMemcpyAsync(&h->sc->dt, &dt, sizeof(double), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
      cudaMemcpyAsync(h->dtlog, &dt, sizeof(double), cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
    return SVE_ERR_CUDA;
  if (h->cfg.precision == SVE_FP64) launch_update<double>(h);
  else launch_update<float>(h);
  if (cudaGetLastError() != cudaSuccess) return SVE_ERR_CUDA;
  rc = wait_status(h);
  h->last_launches = 1;
  h->last_steps = 1;
  return rc;
}

}  // extern "C"
