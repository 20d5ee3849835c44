// sve_noalloc.cu -- sve_step_noalloc: the step loop of libsve for callers
// that cannot allocate device memory.
//
// Who needs it: code that runs where a cudaMalloc is not allowed or not
// possible -- inside a framework whose caching allocator owns the device
// memory (it may have reserved all of it), in a real-time loop that must not
// pay allocation latency or risk an out-of-memory failure mid-run, or in a
// plug-in that is handed device buffers but no allocator.  Such a caller
// passes its own device arrays for the state; every other buffer the step
// needs (padded state, projection, fluctuations, block partials, scalars)
// is carved out of one file-scope device array below.
//
// The array is a static __device__ object: it exists on every GPU that loads
// the library, for the life of the process, whether or not this entry point
// is used.  Its size is SVE_NOALLOC_SCRATCH_BYTES (include/sve.h).
#include <cuda_runtime.h>
#include <stddef.h>
#include <string.h>

#include <mutex>

#include "../../include/sve.h"
#include "sve_device.cuh"

namespace {

// The shared scratch.  In host code this name is only a stand-in for the
// device object: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SVE_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
constexpr int kDtlogEntries = 1024;  // steps per chunk (the per-step dt log lives in the scratch)

std::mutex g_setup_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per
// device (with that device current).
int scratch_address(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SVE_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return SVE_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SVE_ERR_CUDA;
    g_scratch_ptr[dev] = (unsigned char*)p;
  }
  *out = g_scratch_ptr[dev];
  return SVE_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Byte layout of the scratch for one configuration (offsets from the base).
struct Layout {
  size_t fields[13], fx, fy, mpart, sc, dtlog, total;
};

Layout layout_for(const sve::DevParams& P, size_t elem, int nb_cell) {
  Layout L;
  size_t off = 0;
  const size_t next = (size_t)(P.nx + 2) * (size_t)(P.ny + 2);
  for (int k = 0; k < 13; ++k) { L.fields[k] = off; off = align256(off + elem * next); }
  L.fx = off; off = align256(off + 8 * elem * (size_t)P.nfx);
  L.fy = off; off = align256(off + 8 * elem * (size_t)(P.nfy > 0 ? P.nfy : 1));
  L.mpart = off; off = align256(off + 2 * sizeof(double) * (size_t)nb_cell);
  L.sc = off; off = align256(off + sizeof(sve::DevScalars));
  L.dtlog = off; off = align256(off + sizeof(double) * kDtlogEntries);
  L.total = off;
  return L;
}

int status_code(int st) {
  if (st & sve::ST_NAN) return SVE_ERR_NAN;
  if (st & sve::ST_NEG_DEPTH) return SVE_ERR_NEG_DEPTH;
  if (st & sve::ST_RIEMANN) return SVE_ERR_RIEMANN;
  if (st & sve::ST_DT) return SVE_ERR_DT;
  return SVE_OK;
}

template <typename T>
int run(const sve::DevParams& P, unsigned char* base, const Layout& L, int nb_iface, int nb_cell, void* depth,
        void* hu, void* hv, void* zb, int nsteps, double* t_inout, cudaStream_t st) {
  sve::DevState<T> S;
  T** f[13] = {&S.h, &S.hu, &S.hv, &S.z, &S.tau, &S.u, &S.v, &S.pi, &S.omx, &S.omy, &S.ca, &S.cbx, &S.cby};
  for (int k = 0; k < 13; ++k) *f[k] = (T*)(base + L.fields[k]);
  S.fx = (T*)(base + L.fx);
  S.fy = (T*)(base + L.fy);
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
  sve::init_kernel<T><<<(unsigned)sve::cell_blocks(P, sve::kThreads), sve::kThreads, 0, st>>>(P, S, sc, mpart);
  for (int done = 0; done < nsteps;) {
    const int chunk = nsteps - done < kDtlogEntries ? nsteps - done : kDtlogEntries;
    if (cudaMemsetAsync(&sc->call_step, 0, sizeof(int), st) != cudaSuccess) return SVE_ERR_CUDA;
    for (int s = 0; s < chunk; ++s) {
      sve::interface_kernel<T><<<nb_iface, sve::kThreadsStep, 0, st>>>(P, S, sc, dtlog, dtlog, 0);
      sve::cell_kernel<T><<<nb_cell, sve::kThreadsStep, 0, st>>>(P, S, sc, mpart, sve::Mirror<T>{});
    }
    done += chunk;
  }
  if (cudaGetLastError() != cudaSuccess) return SVE_ERR_CUDA;
  for (int k = 0; k < 4; ++k) {
    if (!user[k]) continue;
    const char* src = (const char*)*f[k] + elem * (size_t)(P.ex + 1);
    if (cudaMemcpy2DAsync(user[k], row, src, pitch, row, P.ny, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return SVE_ERR_CUDA;
  }
  sve::DevScalars out;
  if (cudaMemcpyAsync(&out, sc, sizeof(out), cudaMemcpyDeviceToHost, st) != cudaSuccess) return SVE_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return SVE_ERR_CUDA;
  *t_inout = out.t;
  return status_code(out.status);
}

}  // namespace

// Parameter checks and the derived constants are the ones sve_create uses
// (defined in sve_api.cu).
__attribute__((visibility("hidden"))) int sve_internal_validate(const sve_config* c);
__attribute__((visibility("hidden"))) void sve_internal_make_params(const sve_config* c, sve::DevParams* P);

extern "C" int sve_step_noalloc(const sve_config* cfg, void* depth, void* hu, void* hv, void* zb, int nsteps,
                                double* t_inout, void* stream) {
  if (!cfg || !depth || !hu || !zb || !t_inout || nsteps < 0) return SVE_ERR_ARG;
  int rc = sve_internal_validate(cfg);
  if (rc) return rc;
  if (cfg->dim == 2 && !hv) return SVE_ERR_ARG;
  sve::DevParams P;
  sve_internal_make_params(cfg, &P);
  const size_t elem = cfg->precision == SVE_FP64 ? 8 : 4;
  const int nb_iface = (int)sve::iface_blocks(P, sve::kThreadsStep);
  const int nb_cell = (int)sve::cell_blocks(P, sve::kThreadsStep);
  const Layout L = layout_for(P, elem, nb_cell);
  if (L.total > (size_t)SVE_NOALLOC_SCRATCH_BYTES) return SVE_ERR_NOALLOC_SIZE;
  unsigned char* base = nullptr;
  rc = scratch_address(&base);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (cfg->precision == SVE_FP64) return run<double>(P, base, L, nb_iface, nb_cell, depth, hu, hv, zb, nsteps, t_inout, st);
  return run<float>(P, base, L, nb_iface, nb_cell, depth, hu, hv, zb, nsteps, t_inout, st);
}
