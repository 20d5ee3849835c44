// sve_noalloc.cu -- sve_step_noalloc: the step loop of libsve for callers
// that cannot allocate device memory.
//
// Who needs it: code that runs where a cudaMalloc is not allowed or not
// possible -- inside a framework whose caching allocator owns the device
// memory (it may have reserved all of it), in a real-time loop that must not
// pay allocation latency or risk an out-of-memory failure mid-run, or in a
// plug-in that is handed device buffers but no allocator.  Such a caller
// passes its own device arrays for the state; every other buffer the step
// needs (padded state, projection or net fluctuations, interface
// fluctuations, block partials, scalars) is carved out of one file-scope
// device array below.
//
// The kernels are those of the regular entry points for the configuration:
// the two-kernel step (interface_kernel + cell_kernel) in FP64 and in 1D,
// the fused FP32 stencil (march_kernel + apply_kernel) for the FP32 state in
// 2D.
//
// The array is a static __device__ object: it exists on every GPU that loads
// the library, for the life of the process, whether or not this entry point
// is used.  Its size is SVE_NOALLOC_SCRATCH_BYTES (include/sve.h).
#include <cuda_runtime.h>
#include <stddef.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "../../include/sve.h"
#include "sve_device.cuh"
#include "sve_fused.cuh"
#include "sve_march.cuh"

// Parameter checks, derived constants and status codes are the ones the
// regular entry points use (defined in sve_api.cu).
__attribute__((visibility("hidden"))) int sve_internal_validate(const sve_config* c);
__attribute__((visibility("hidden"))) void sve_internal_make_params(const sve_config* c, sve::DevParams* P);
__attribute__((visibility("hidden"))) int sve_internal_status_code(int st);
__attribute__((visibility("hidden"))) bool sve_internal_has_external(const sve_config* c);

namespace {

// The shared scratch.  In host code this name is only a stand-in for the
// device object: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SVE_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
constexpr int kDtlogEntries = 1024;  // steps per chunk (the per-step dt log lives in the scratch)

std::mutex g_setup_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {};
int g_nsm[kMaxDevices] = {};          // SMs of the device

// Device address of the scratch on the current device, and the launch facts
// the fused FP32 step needs, looked up once per device (with that device
// current).
int device_setup(int* dev_out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SVE_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return SVE_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SVE_ERR_CUDA;
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
      return SVE_ERR_CUDA;
    g_nsm[dev] = nsm;
    g_scratch_ptr[dev] = (unsigned char*)p;
  }
  *dev_out = dev;
  return SVE_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Launch shape of one call: the two-kernel step (blocks of the interface and
// cell kernels) or the fused FP32 stencil (the strips of the solve pass, the
// apply pass's 2D grid); nmpart = block partials the largest pass writes.
struct Shape {
  bool fused;
  int nb_iface, nb_cell;                 // two-kernel step
  sve::MarchShape march;                 // fused: solve pass
  int agx, agy;                          // fused: apply grid
  size_t nmpart;
};

Shape shape_for(const sve::DevParams& P, bool fused, int nsm) {
  Shape S = {};
  S.fused = fused;
  const size_t init_blocks = (size_t)sve::cell_blocks(P, sve::kThreads);
  if (!fused) {
    S.nb_iface = (int)sve::iface_blocks(P, sve::kThreadsStep);
    S.nb_cell = (int)sve::cell_blocks(P, sve::kThreadsStep);
    S.nmpart = std::max(init_blocks, (size_t)S.nb_cell);
  } else {
    S.march = sve::march_shape(P, nsm);
    S.agx = (P.nx + sve::kAThreads - 1) / sve::kAThreads;
    S.agy = std::min(P.ny, std::max(1, (nsm * (2048 / sve::kAThreads) + S.agx - 1) / S.agx));
    S.nmpart = std::max(init_blocks, (size_t)S.agx * (size_t)S.agy);
  }
  return S;
}

// Byte layout of the scratch for one configuration (offsets from the base):
// 13 padded fields (state + projection: the state upload's init_kernel
// writes all of them), then the fluctuation planes of the two-kernel step or
// the 4 planes of net fluctuations of the fused step.
struct Layout {
  size_t fields[13], fx, fy, net, mpart, sc, dtlog, total;
};

Layout layout_for(const sve::DevParams& P, size_t elem, const Shape& S) {
  Layout L = {};
  size_t off = 0;
  const size_t next = (size_t)(P.nx + 2) * (size_t)(P.ny + 2);
  for (int k = 0; k < 13; ++k) { L.fields[k] = off; off = align256(off + elem * next); }
  if (!S.fused) {
    L.fx = off; off = align256(off + 8 * elem * (size_t)P.nfx);
    L.fy = off; off = align256(off + 8 * elem * (size_t)(P.nfy > 0 ? P.nfy : 1));
  } else {
    L.net = off; off = align256(off + 4 * elem * (size_t)P.nx * (size_t)P.ny);
  }
  L.mpart = off; off = align256(off + 2 * sizeof(double) * S.nmpart);
  L.sc = off; off = align256(off + sizeof(sve::DevScalars));
  L.dtlog = off; off = align256(off + sizeof(double) * kDtlogEntries);
  L.total = off;
  return L;
}

}  // namespace

namespace {

// The latched device status, read after the stream's work so far (one small
// copy and a wait).
int read_status(const sve::DevScalars* sc, cudaStream_t st, double* t_out) {
  sve::DevScalars host;
  if (cudaMemcpyAsync(&host, sc, sizeof(host), cudaMemcpyDeviceToHost, st) != cudaSuccess) return SVE_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return SVE_ERR_CUDA;
  if (t_out) *t_out = host.t;
  return sve_internal_status_code(host.status);
}

template <typename T>
int run(const sve::DevParams& P, unsigned char* base, const Layout& L, const Shape& SH, void* depth, void* hu,
        void* hv, void* zb, int nsteps, double* t_inout, cudaStream_t st) {
  sve::DevState<T> S = {};
  T** f[13] = {&S.h, &S.hu, &S.hv, &S.z, &S.tau, &S.u, &S.v, &S.pi, &S.omx, &S.omy, &S.ca, &S.cbx, &S.cby};
  for (int k = 0; k < 13; ++k) *f[k] = (T*)(base + L.fields[k]);
  if (!SH.fused) {
    S.fx = (T*)(base + L.fx);
    S.fy = (T*)(base + L.fy);
  }
  double* mpart = (double*)(base + L.mpart);
  sve::DevScalars* sc = (sve::DevScalars*)(base + L.sc);
  double* dtlog = (double*)(base + L.dtlog);
  const size_t elem = sizeof(T);
  const size_t row = elem * (size_t)P.nx;
  const size_t pitch = elem * (size_t)P.ex;
  const size_t next = (size_t)(P.nx + 2) * (size_t)(P.ny + 2);

  // the scratch keeps the previous call's contents: clear what must start
  // at zero (scalars and counters; hv in 1D) before use
  if (cudaMemsetAsync(sc, 0, sizeof(sve::DevScalars), st) != cudaSuccess) return SVE_ERR_CUDA;
  if (P.dim == 1 && cudaMemsetAsync(S.hv, 0, elem * next, st) != cudaSuccess) return SVE_ERR_CUDA;
  if (cudaMemcpyAsync(&sc->t, t_inout, sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return SVE_ERR_CUDA;
  void* user[4] = {depth, hu, P.dim == 2 ? hv : nullptr, zb};
  for (int k = 0; k < 4; ++k) {
    if (!user[k]) continue;
    char* dst = (char*)*f[k] + elem * (size_t)(P.ex + 1);
    if (cudaMemcpy2DAsync(dst, pitch, user[k], row, row, P.ny, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return SVE_ERR_CUDA;
  }
  // ghosts, projection (two-kernel step) and the checks of the input state;
  // a bad input is reported before any step, the caller's arrays untouched
  sve::init_kernel<T><<<(unsigned)sve::cell_blocks(P, sve::kThreads), sve::kThreads, 0, st>>>(P, S, sc, mpart);
  if (cudaGetLastError() != cudaSuccess) return SVE_ERR_CUDA;
  int rc = read_status(sc, st, nullptr);
  if (rc) return rc;
  sve::StateBuf<T> B = {S.h, S.hu, S.hv, S.z};
  sve::NetFluct<T> D = {};
  if (SH.fused) {
    const size_t ncell = (size_t)P.nx * (size_t)P.ny;
    D.h = (T*)(base + L.net); D.hu = D.h + ncell; D.hv = D.hu + ncell; D.z = D.hv + ncell;
  }
  for (int done = 0; done < nsteps;) {
    const int chunk = nsteps - done < kDtlogEntries ? nsteps - done : kDtlogEntries;
    if (cudaMemsetAsync(&sc->call_step, 0, sizeof(int), st) != cudaSuccess) return SVE_ERR_CUDA;
    for (int s = 0; s < chunk; ++s) {
      if constexpr (sizeof(T) == 4) {
        if (SH.fused) {
          sve::march_kernel<T><<<SH.march.blocks, sve::kMThreads, 0, st>>>(P, B, D, sc, dtlog, dtlog, 0, SH.march.strips,
                                                                          SH.march.rows, SH.march.tasks);
          sve::apply_kernel<T><<<dim3(SH.agx, SH.agy), sve::kAThreads, 0, st>>>(P, B, B, D, sc, mpart,
                                                                                sve::Mirror<T>{});
          continue;
        }
      }
      sve::interface_kernel<T><<<SH.nb_iface, sve::kThreadsStep, 0, st>>>(P, S, sc, dtlog, dtlog, 0);
      sve::cell_kernel<T><<<SH.nb_cell, sve::kThreadsStep, 0, st>>>(P, S, sc, mpart, sve::Mirror<T>{});
    }
    done += chunk;
  }
  if (cudaGetLastError() != cudaSuccess) return SVE_ERR_CUDA;
  // the steps' latched status first: on an error the caller's arrays keep
  // their input
  double t_new = *t_inout;
  rc = read_status(sc, st, &t_new);
  if (rc) return rc;
  for (int k = 0; k < 4; ++k) {
    if (!user[k]) continue;
    const char* src = (const char*)*f[k] + elem * (size_t)(P.ex + 1);
    if (cudaMemcpy2DAsync(user[k], row, src, pitch, row, P.ny, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return SVE_ERR_CUDA;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return SVE_ERR_CUDA;
  *t_inout = t_new;
  return SVE_OK;
}

}  // namespace

extern "C" int sve_step_noalloc(const sve_config* cfg, void* depth, void* hu, void* hv, void* zb, int nsteps,
                                double* t_inout, void* stream) {
  if (!cfg || !depth || !hu || !zb || !t_inout || nsteps < 0) return SVE_ERR_ARG;
  int rc = sve_internal_validate(cfg);
  if (rc) return rc;
  if ((cfg->dim == 2 && !hv) || sve_internal_has_external(cfg)) return SVE_ERR_ARG;
  sve::DevParams P;
  sve_internal_make_params(cfg, &P);
  int dev = 0;
  rc = device_setup(&dev);
  if (rc) return rc;
  const bool fused = cfg->precision == SVE_FP32 && cfg->dim == 2;
  const Shape SH = shape_for(P, fused, g_nsm[dev]);
  const size_t elem = cfg->precision == SVE_FP64 ? 8 : 4;
  const Layout L = layout_for(P, elem, SH);
  if (L.total > (size_t)SVE_NOALLOC_SCRATCH_BYTES) return SVE_ERR_NOALLOC_SIZE;
  unsigned char* base = g_scratch_ptr[dev];
  cudaStream_t st = (cudaStream_t)stream;
  if (cfg->precision == SVE_FP64) return run<double>(P, base, L, SH, depth, hu, hv, zb, nsteps, t_inout, st);
  return run<float>(P, base, L, SH, depth, hu, hv, zb, nsteps, t_inout, st);
}
