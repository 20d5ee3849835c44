// sve_api.cu -- host side of libsve: handle, device memory, state transfer,
// the step loop (CUDA graphs of step pairs) and error reporting.  The C ABI is
// declared in include/sve.h.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "../../include/sve.h"
#include "sve_device.cuh"
#include "sve_fused.cuh"
#include "sve_march.cuh"
#include "sve_persist.cuh"
#include "sve_handle.h"

using sve::DevParams;
using sve::DevScalars;
using sve::DevState;

namespace {
constexpr int kGraphSteps = 16;  // steps per captured graph
}  // namespace

namespace {

#define SVE_TRY(expr)                         \
  do {                                        \
    cudaError_t _e = (expr);                  \
    if (_e != cudaSuccess) return SVE_ERR_CUDA; \
  } while (0)

int status_to_code(int st) {
  if (st & sve::ST_NAN) return SVE_ERR_NAN;
  if (st & sve::ST_NEG_DEPTH) return SVE_ERR_NEG_DEPTH;
  if (st & sve::ST_RIEMANN) return SVE_ERR_RIEMANN;
  if (st & sve::ST_DT) return SVE_ERR_DT;
  if (st & sve::ST_SYNC) return SVE_ERR_SYNC;
  return SVE_OK;
}

int validate(const sve_config* c) {
  if (!c) return SVE_ERR_ARG;
  if (c->dim != 1 && c->dim != 2) return SVE_ERR_ARG;
  if (c->nx < 1 || c->ny < 1 || (c->dim == 1 && c->ny != 1)) return SVE_ERR_ARG;
  if ((long long)c->nx * c->ny > (1LL << 31) - 1) return SVE_ERR_ARG;
  if (!(c->lx > 0) || (c->dim == 2 && !(c->ly > 0)) || !(c->g > 0) || !(c->cfl > 0)) return SVE_ERR_ARG;
  if (c->precision != SVE_FP64 && c->precision != SVE_FP32) return SVE_ERR_ARG;
  if (c->bedload < SVE_GRASS || c->bedload > SVE_CAMENEN) return SVE_ERR_ARG;
  if (c->bedload == SVE_GRASS && (!(c->m_g >= 1.0) || !(c->m_g <= 4.0) || !(c->A_g >= 0.0))) return SVE_ERR_ARG;
  if (c->friction < SVE_FRIC_NONE || c->friction > SVE_FRIC_STRICKLER) return SVE_ERR_ARG;
  if (c->bedload != SVE_GRASS && (c->friction == SVE_FRIC_NONE || !(c->s > 1.0) || !(c->d_s > 0.0))) return SVE_ERR_ARG;
  if (c->friction == SVE_FRIC_STRICKLER && !(c->K_st > 0)) return SVE_ERR_ARG;
  if (c->friction == SVE_FRIC_DARCY && !(c->f_dw >= 0)) return SVE_ERR_ARG;
  const int nsides = c->dim == 2 ? 4 : 2;
  for (int s = 0; s < nsides; ++s)
    if (c->bc[s] < SVE_BC_PERIODIC || c->bc[s] > SVE_BC_EXTERNAL) return SVE_ERR_ARG;
  if ((c->bc[0] == SVE_BC_PERIODIC) != (c->bc[1] == SVE_BC_PERIODIC)) return SVE_ERR_ARG;
  if (c->dim == 2 && (c->bc[2] == SVE_BC_PERIODIC) != (c->bc[3] == SVE_BC_PERIODIC)) return SVE_ERR_ARG;
  if (!(c->kappa_a > 1.0) || !(c->beta_min > 0.0) || !(c->gamma_z >= 0.0)) return SVE_ERR_ARG;
  if (!(c->newton_tol > 0.0) || c->newton_maxit < 1 || c->newton_maxit > 1000) return SVE_ERR_ARG;
  return SVE_OK;
}

void make_params(const sve_config* c, DevParams* P) {
  memset(P, 0, sizeof(*P));
  P->dim = c->dim;
  P->nx = c->nx;
  P->ny = c->dim == 2 ? c->ny : 1;
  P->ex = c->nx + 2;
  P->dx = c->lx / c->nx;
  P->dy = c->dim == 2 ? c->ly / c->ny : 1.0;
  P->inv_dx = 1.0 / P->dx;
  P->inv_dy = 1.0 / P->dy;
  P->g = c->g;
  P->inv_2g = 1.0 / (2.0 * c->g);
  P->cfl = c->cfl;
  P->bedload = c->bedload;
  P->A_g = c->A_g;
  P->m_g = c->m_g;
  P->m_int = (c->m_g == 1.0 || c->m_g == 2.0 || c->m_g == 3.0 || c->m_g == 4.0) ? (int)c->m_g : 0;
  const double sm1 = c->s - 1.0;
  P->qs_scale = sqrt(sm1 * c->g * c->d_s * c->d_s * c->d_s);
  if (c->friction == SVE_FRIC_DARCY) {
    P->mpm_alpha = c->f_dw / (8.0 * c->g * sm1 * c->d_s);
  } else if (c->friction == SVE_FRIC_STRICKLER) {
    const double n = 1.0 / c->K_st;
    P->mpm_alpha = (n * n) / (sm1 * c->d_s);
  }
  P->tau_cr = c->tau_cr;
  P->friction = c->friction;
  if (c->friction == SVE_FRIC_DARCY) { P->fric_c = c->f_dw / 8.0; P->fric_coef = c->f_dw; }
  else if (c->friction == SVE_FRIC_STRICKLER) { P->fric_c = c->g / (c->K_st * c->K_st); P->fric_coef = c->K_st; }
  for (int s = 0; s < 4; ++s) P->bc[s] = c->bc[s];
  P->q_in = c->q_in;
  P->h_in = c->h_in;
  P->kappa_a = c->kappa_a;
  P->beta_min = c->beta_min;
  P->gamma_z = c->gamma_z;
  P->newton_tol = c->newton_tol;
  P->newton_maxit = c->newton_maxit;
  P->two_g = 2.0 * c->g;
  P->two_g_gamma = 2.0 * c->g * c->gamma_z;
  P->nfx = (long long)(P->nx + 1) * P->ny;
  P->nfy = P->dim == 2 ? (long long)P->nx * (P->ny + 1) : 0;
  P->f.g = (float)P->g;
  P->f.inv_2g = (float)P->inv_2g;
  P->f.A_g = (float)P->A_g;
  P->f.m_g = (float)P->m_g;
  P->f.qs_scale = (float)P->qs_scale;
  P->f.mpm_alpha = (float)P->mpm_alpha;
  P->f.tau_cr = (float)P->tau_cr;
  P->f.fric_c = (float)P->fric_c;
  P->f.q_in = (float)P->q_in;
  P->f.h_in = (float)P->h_in;
  P->f.kappa_a = (float)P->kappa_a;
  P->f.beta_min = (float)P->beta_min;
  P->f.gamma_z = (float)P->gamma_z;
  P->f.newton_tol = (float)P->newton_tol;
  P->f.two_g = (float)P->two_g;
  P->f.two_g_gamma = (float)P->two_g_gamma;
}

// The parameters of the step's kernels: the configuration's, or for the
// splitting scheme its shallow-water step's (transport switched off).
const DevParams& step_params(const sve_handle* h) { return h->scheme ? h->P_sw : h->P; }

template <typename T>
void launch_step(sve_handle* h, cudaStream_t st, int fixed, cudaEvent_t* ev, const void* const* mirror) {
  DevState<T> S = state_of<T>(h);
  sve::Mirror<T> out{};
  if (mirror) out = {(T*)mirror[0], (T*)mirror[1], (T*)mirror[2], (T*)mirror[3]};
  const int nt = h->nt;
  const DevParams& PS = step_params(h);
  const unsigned nbi = (unsigned)sve::iface_blocks(h->P, nt), nbc = (unsigned)sve::cell_blocks(h->P, nt);
  const bool split = std::is_same<T, double>::value && h->scheme;
  if (split) cudaMemcpyAsync(h->zsave, h->fields[3], sizeof(double) * (size_t)h->next, cudaMemcpyDeviceToDevice, st);
  if (ev) cudaEventRecord(ev[0], st);
  if (nt == sve::kThreadsNarrow)
    sve::interface_kernel<T, sve::kThreadsNarrow><<<nbi, nt, 0, st>>>(PS, S, h->sc, h->fixed, h->dtlog, fixed);
  else if (nt == sve::kThreadsStep)
    sve::interface_kernel<T, sve::kThreadsStep><<<nbi, nt, 0, st>>>(PS, S, h->sc, h->fixed, h->dtlog, fixed);
  else
    sve::interface_kernel<T, sve::kThreads><<<nbi, nt, 0, st>>>(PS, S, h->sc, h->fixed, h->dtlog, fixed);
  if (ev) cudaEventRecord(ev[1], st);
  if (nt == sve::kThreadsNarrow)
    sve::cell_kernel<T, sve::kThreadsNarrow><<<nbc, nt, 0, st>>>(PS, S, h->sc, h->mpart, out);
  else if (nt == sve::kThreadsStep)
    sve::cell_kernel<T, sve::kThreadsStep><<<nbc, nt, 0, st>>>(PS, S, h->sc, h->mpart, out);
  else
    sve::cell_kernel<T, sve::kThreads><<<nbc, nt, 0, st>>>(PS, S, h->sc, h->mpart, out);
  if constexpr (std::is_same<T, double>::value) {
    if (split) {
      // the Exner update of the held bed with the configured transport law
      if (nt == sve::kThreadsNarrow)
        sve::exner_kernel<sve::kThreadsNarrow><<<nbc, nt, 0, st>>>(h->P, S, h->zsave, h->sc, h->mpart);
      else if (nt == sve::kThreadsStep)
        sve::exner_kernel<sve::kThreadsStep><<<nbc, nt, 0, st>>>(h->P, S, h->zsave, h->sc, h->mpart);
      else
        sve::exner_kernel<sve::kThreads><<<nbc, nt, 0, st>>>(h->P, S, h->zsave, h->sc, h->mpart);
    }
  }
  if (ev) cudaEventRecord(ev[2], st);
}

// FP32 state in 2D: the solve pass (column strips marching over rows,
// fluctuations in registers, net fluctuation per cell out, time step from
// the solves) and the in-place apply pass.
void launch_fused_step(sve_handle* h, cudaStream_t st, int fixed, cudaEvent_t* ev, const void* const* mirror) {
  sve::StateBuf<float> B;
  B.h = (float*)h->fields[0]; B.hu = (float*)h->fields[1]; B.hv = (float*)h->fields[2]; B.z = (float*)h->fields[3];
  const size_t ncell = (size_t)h->P.nx * (size_t)h->P.ny;
  sve::NetFluct<float> D;  // in the fluctuation planes of the two-kernel form (8 (nx+1) ny >= 4 nx ny floats)
  D.h = (float*)h->fx; D.hu = D.h + ncell; D.hv = D.hu + ncell; D.z = D.hv + ncell;
  const sve::MarchShape& M = h->march;
  if (ev) cudaEventRecord(ev[0], st);
  sve::march_kernel<float><<<M.blocks, sve::kMThreads, 0, st>>>(h->P, B, D, h->sc, h->fixed, h->dtlog, fixed,
                                                                M.strips, M.rows, M.tasks);
  if (ev) cudaEventRecord(ev[1], st);
  sve::Mirror<float> out{};
  if (mirror) out = {(float*)mirror[0], (float*)mirror[1], (float*)mirror[2], (float*)mirror[3]};
  sve::apply_kernel<float><<<dim3(h->agx, h->agy), sve::kAThreads, 0, st>>>(h->P, B, B, D, h->sc, h->mpart, out);
  if (ev) cudaEventRecord(ev[2], st);
}

// The carried update within a call of n steps (FP32 state in 2D): step 0's
// solve pass on U^0 in the handle's state buffer; step k >= 1's solve pass
// applies step k - 1's update as it reads U^{k-1} from buffer (k - 1) % 2 and
// the net fluctuations from half (k - 1) % 2 of the fluctuation planes,
// storing U^k into the other buffer and its own net fluctuations into the
// other half; after step n - 1 the apply pass takes U^{n-1} and the last
// update into the handle's state buffer (ghosts, checks, mass sums).  Every
// state and time step equals the one-step-at-a-time sequence bit for bit.
sve::StateBuf<float> fused_buf(const sve_handle* h, int p) {
  void* const* f = p ? h->alt : h->fields;
  return {(float*)f[0], (float*)f[1], (float*)f[2], (float*)f[3]};
}
sve::NetFluct<float> fused_dF(const sve_handle* h, int p) {
  const size_t ncell = (size_t)h->P.nx * (size_t)h->P.ny;
  float* b = (float*)h->fx + (size_t)p * 4 * ncell;  // 8 (nx + 1) ny >= 8 nx ny floats
  return {b, b + ncell, b + 2 * ncell, b + 3 * ncell};
}

// The solve pass of step k of a carried call.
void launch_carried_march(sve_handle* h, cudaStream_t st, int fixed, int k, cudaEvent_t* ev) {
  const sve::MarchShape& M = h->march;
  if (ev) cudaEventRecord(ev[0], st);
  if (k == 0) {
    sve::march_kernel<float><<<M.blocks, sve::kMThreads, 0, st>>>(h->P, fused_buf(h, 0), fused_dF(h, 0), h->sc,
                                                                  h->fixed, h->dtlog, fixed, M.strips, M.rows,
                                                                  M.tasks);
  } else {
    const int q = (k - 1) & 1;
    sve::march_kernel<float><<<M.blocks, sve::kMThreads, 0, st>>>(
        h->P, fused_buf(h, q), fused_dF(h, 1 - q), h->sc, h->fixed, h->dtlog, fixed, M.strips, M.rows, M.tasks, 1,
        fused_buf(h, 1 - q), fused_dF(h, q));
  }
  if (ev) {
    cudaEventRecord(ev[1], st);
    cudaEventRecord(ev[2], st);
  }
}

// The apply pass after the last solve pass (step n - 1) of a carried call.
void launch_carried_apply(sve_handle* h, cudaStream_t st, int n, cudaEvent_t* ev, const void* const* mirror) {
  const int q = (n - 1) & 1;
  sve::Mirror<float> out{};
  if (mirror) out = {(float*)mirror[0], (float*)mirror[1], (float*)mirror[2], (float*)mirror[3]};
  if (ev) {
    cudaEventRecord(ev[0], st);
    cudaEventRecord(ev[1], st);
  }
  sve::apply_kernel<float><<<dim3(h->agx, h->agy), sve::kAThreads, 0, st>>>(
      h->P, fused_buf(h, q), fused_buf(h, 0), fused_dF(h, q), h->sc, h->mpart, out);
  if (ev) cudaEventRecord(ev[2], st);
}

// mirror: null, or four row-major destinations (device-accessible) that the
// step's cell update also writes the new interior state to.
// One record of the per-step history ring after a step: (t, dt, mass_h,
// mass_z, Sx, Sy) -- the masses from the step's per-block partials, summed
// as mass_kernel sums them.
__global__ void __launch_bounds__(sve::kThreads) history_kernel(DevParams P, DevScalars* sc, const double* mpart,
                                                                double* hist, int cap) {
  __shared__ double sh[2 * (sve::kThreads / 32)];
  double a, b;
  sve::reduce_partials<sve::kThreads>(mpart, sc->mass_parts, a, b, sh);
  if (threadIdx.x != 0) return;
  const double cell = P.dx * (P.dim == 2 ? P.dy : 1.0);
  double* r = hist + 6 * (size_t)(sc->hist_count % (unsigned long long)cap);
  r[0] = sc->t;
  r[1] = sc->dt;
  r[2] = a * cell;
  r[3] = b * cell;
  r[4] = sc->Sx;
  r[5] = P.dim == 2 ? sc->Sy : 0.0;
  sc->hist_count += 1;
}

void launch_step_any(sve_handle* h, cudaStream_t st, int fixed, cudaEvent_t* ev = nullptr,
                     const void* const* mirror = nullptr) {
  if (h->cfg.precision == SVE_FP64) launch_step<double>(h, st, fixed, ev, mirror);
  else if (h->fused) launch_fused_step(h, st, fixed, ev, mirror);
  else launch_step<float>(h, st, fixed, ev, mirror);
  if (h->hist_cap > 0) history_kernel<<<1, sve::kThreads, 0, st>>>(h->P, h->sc, h->mpart, h->hist, h->hist_cap);
}

// Three events for one profiled step or pass (grown on demand); kind: which
// intervals count (bit 0: solve pass, bit 1: update pass).
cudaEvent_t* next_events(sve_handle* h, unsigned char kind = 3) {
  while (h->events.size() < h->events_used + 3) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    h->events.push_back(e);
  }
  if (h->ev_kind.size() < h->events.size() / 3) h->ev_kind.resize(h->events.size() / 3);
  h->ev_kind[h->events_used / 3] = kind;
  cudaEvent_t* ev = &h->events[h->events_used];
  h->events_used += 3;
  return ev;
}

// Fold the recorded events into the per-kernel totals (waits for them).
int drain_events(sve_handle* h) {
  for (size_t k = 0; k + 3 <= h->events_used; k += 3) {
    float a = 0.f, b = 0.f;
    if (cudaEventSynchronize(h->events[k + 2]) != cudaSuccess) return SVE_ERR_CUDA;
    if (cudaEventElapsedTime(&a, h->events[k], h->events[k + 1]) != cudaSuccess) return SVE_ERR_CUDA;
    if (cudaEventElapsedTime(&b, h->events[k + 1], h->events[k + 2]) != cudaSuccess) return SVE_ERR_CUDA;
    const unsigned char kind = h->ev_kind[k / 3];
    if (kind & 1) {
      h->prof_ms[0] += a;
      h->prof_launches[0] += 1;
    }
    if (kind & 2) {
      h->prof_ms[1] += b;
      h->prof_launches[1] += 1;
    }
  }
  h->events_used = 0;
  return SVE_OK;
}

int ensure_capacity(double** buf, int* cap, int n) {
  if (n <= *cap) return SVE_OK;
  int ncap = n > 2 * *cap ? n : 2 * *cap;
  double* nb = nullptr;
  if (cudaMalloc(&nb, sizeof(double) * (size_t)ncap) != cudaSuccess) return SVE_ERR_OOM;
  if (*buf) cudaFree(*buf);
  *buf = nb;
  *cap = ncap;
  return SVE_OK;
}

// Whether calls of several steps carry the FP32 2D update into the next
// solve pass (not while per-step records are kept: those need each step's
// mass sums).
bool carrying(const sve_handle* h) { return h->carry && h->hist_cap == 0; }

// kGraphSteps steps: the two-kernel or fused step, or, for the carried
// update, kGraphSteps carried solve passes from buffer 0 (steps k = 1, 3,
// ... of a call: kGraphSteps is even, so every such graph starts there).
int get_graph(sve_handle* h, int fixed, cudaGraphExec_t* out) {
  cudaGraphExec_t& G = h->graph[fixed ? 1 : 0];
  if (!G) {
    cudaGraph_t g = nullptr;
    SVE_TRY(cudaStreamBeginCapture(h->capture, cudaStreamCaptureModeThreadLocal));
    for (int s = 0; s < kGraphSteps; ++s) {
      if (carrying(h)) launch_carried_march(h, h->capture, fixed, s + 1, nullptr);
      else launch_step_any(h, h->capture, fixed);
    }
    cudaError_t e = cudaStreamEndCapture(h->capture, &g);
    if (e != cudaSuccess) return SVE_ERR_CUDA;
    e = cudaGraphInstantiate(&G, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { G = nullptr; return SVE_ERR_CUDA; }
  }
  *out = G;
  return SVE_OK;
}

void drop_graphs(sve_handle* h) {
  for (auto& G : h->graph) {
    if (G) cudaGraphExecDestroy(G);
    G = nullptr;
  }
}

// Whether steps run as persistent cooperative launches (opt-in: measured no
// faster than the two kernels from CUDA graphs, whose launches overlap the
// steps' FP64 latency chains).
bool use_persistent(const sve_handle* h) {
  return h->persist_ok && !h->profiling && h->persist_mode == 1 && !h->scheme && h->hist_cap == 0;
}

constexpr int kPersistChunk = 4096;  // steps per persistent launch

// One persistent cooperative launch of nsteps steps (expected / polls: the
// barrier's arrivals and wait bound).
int launch_persistent(sve_handle* h, int nsteps, int fixed, unsigned int expected, long long polls) {
  SVE_TRY(cudaMemsetAsync(h->ps, 0, sizeof(sve::PersistScratch), h->stream));
  void* args[11];
  DevParams P = h->P;
  int fx = fixed, ns = nsteps;
  const double* fd = h->fixed;
  double* dl = h->dtlog;
  double* mp = h->mpart;
  sve::DevScalars* sc = h->sc;
  sve::PersistScratch* ps = h->ps;
  if (h->cfg.precision == SVE_FP64) {
    DevState<double> S = state_of<double>(h);
    void* a[11] = {&P, &S, &sc, &ps, &fd, &dl, &fx, &ns, &mp, &expected, &polls};
    for (int k = 0; k < 11; ++k) args[k] = a[k];
    SVE_TRY(cudaLaunchCooperativeKernel((const void*)sve::persistent_kernel<double>, dim3(h->pgrid),
                                        dim3(sve::kPersistThreads), args, 0, h->stream));
  } else {
    DevState<float> S = state_of<float>(h);
    void* a[11] = {&P, &S, &sc, &ps, &fd, &dl, &fx, &ns, &mp, &expected, &polls};
    for (int k = 0; k < 11; ++k) args[k] = a[k];
    SVE_TRY(cudaLaunchCooperativeKernel((const void*)sve::persistent_kernel<float>, dim3(h->pgrid),
                                        dim3(sve::kPersistThreads), args, 0, h->stream));
  }
  return SVE_OK;
}

// Enqueue nsteps steps on the handle's stream (graphs of kGraphSteps steps
// where possible; single launches with events when profiling; persistent
// cooperative launches of up to kPersistChunk steps on small grids).
int enqueue_steps(sve_handle* h, int nsteps, int fixed, const void* const* mirror = nullptr) {
  if (!h->has_state) return SVE_ERR_STATE;
  double* old = h->dtlog;
  int rc = ensure_capacity(&h->dtlog, &h->dtlog_cap, nsteps > 0 ? nsteps : 1);
  if (rc) return rc;
  if (h->dtlog != old) drop_graphs(h);  // graphs hold the dtlog pointer
  SVE_TRY(cudaMemsetAsync(&h->sc->call_step, 0, sizeof(int), h->stream));
  int done = 0;
  long long launches = 0;
  if (use_persistent(h)) {
    // with a mirror the last step is a single two-kernel step
    const int np = mirror ? nsteps - 1 : nsteps;
    for (; done < np; done += kPersistChunk) {
      rc = launch_persistent(h, std::min(kPersistChunk, np - done), fixed, (unsigned int)h->pgrid,
                             sve::kBarrierPolls);
      if (rc) return rc;
      ++launches;
    }
    done = np;
    if (done < nsteps) {
      launch_step_any(h, h->stream, fixed, nullptr, mirror);
      launches += 2;
    }
    SVE_TRY(cudaGetLastError());
    h->last_launches = launches;
    h->last_steps = nsteps;
    return SVE_OK;
  }
  if (carrying(h) && nsteps > 1) {
    // the carried update: step 0, steps 1 .. n - 1 (graphs of kGraphSteps
    // from step 1 on), the apply pass (one step: the plain step below)
    int k = 1;
    cudaEvent_t* ev = h->profiling ? next_events(h, 1) : nullptr;
    if (h->profiling && !ev) return SVE_ERR_CUDA;
    launch_carried_march(h, h->stream, fixed, 0, ev);
    if (nsteps - 1 >= kGraphSteps && !h->profiling) {
      cudaGraphExec_t ex;
      rc = get_graph(h, fixed, &ex);
      if (rc) return rc;
      for (; k + kGraphSteps <= nsteps; k += kGraphSteps) SVE_TRY(cudaGraphLaunch(ex, h->stream));
    }
    for (; k < nsteps; ++k) {
      ev = h->profiling ? next_events(h, 1) : nullptr;
      if (h->profiling && !ev) return SVE_ERR_CUDA;
      launch_carried_march(h, h->stream, fixed, k, ev);
    }
    ev = h->profiling ? next_events(h, 2) : nullptr;
    if (h->profiling && !ev) return SVE_ERR_CUDA;
    launch_carried_apply(h, h->stream, nsteps, ev, mirror);
    SVE_TRY(cudaGetLastError());
    h->last_launches = (long long)nsteps + 1;
    h->last_steps = nsteps;
    return SVE_OK;
  }
  // with a mirror the last step is a single launch (the graphs write no mirror)
  const int graphed = mirror ? nsteps - 1 : nsteps;
  if (graphed >= kGraphSteps && !h->profiling) {
    cudaGraphExec_t ex;
    rc = get_graph(h, fixed, &ex);
    if (rc) return rc;
    for (; done + kGraphSteps <= graphed; done += kGraphSteps) SVE_TRY(cudaGraphLaunch(ex, h->stream));
  }
  for (; done < nsteps; ++done) {
    cudaEvent_t* ev = h->profiling ? next_events(h) : nullptr;
    if (h->profiling && !ev) return SVE_ERR_CUDA;
    launch_step_any(h, h->stream, fixed, ev, done == nsteps - 1 ? mirror : nullptr);
  }
  SVE_TRY(cudaGetLastError());
  h->last_launches = 2LL * nsteps;
  h->last_steps = nsteps;
  return SVE_OK;
}

// Mass sums of the last step (or upload) from its per-block partials, in a
// fixed order (one block; launched when the diagnostics are read).
__global__ void __launch_bounds__(sve::kThreads) mass_kernel(DevParams P, DevScalars* sc, const double* mpart) {
  __shared__ double sh[2 * (sve::kThreads / 32)];
  double a, b;
  sve::reduce_partials<sve::kThreads>(mpart, sc->mass_parts, a, b, sh);
  if (threadIdx.x == 0) {
    const double cell = P.dx * (P.dim == 2 ? P.dy : 1.0);
    sc->mass_h = a * cell;
    sc->mass_z = b * cell;
  }
}

int auto_block_size(const sve_handle* h) {
  return sve::iface_blocks(h->P, sve::kThreads) < 2LL * h->nsm ? sve::kThreadsNarrow : sve::kThreadsStep;
}

int wait_status(sve_handle* h) {
  DevScalars s;
  SVE_TRY(cudaMemcpyAsync(&s, h->sc, sizeof(s), cudaMemcpyDeviceToHost, h->stream));
  SVE_TRY(cudaStreamSynchronize(h->stream));
  h->last_t = s.t;
  return status_to_code(s.status);
}

// Projection, checks, ghosts and mass partials of the cells k0..k1-1 (a
// band of whole rows) after an upload: init_kernel for a part of the grid.
// Blocks b0.. of nb_total over all bands write the partials; the last of
// all of them records the partial count.
template <typename T>
__global__ void __launch_bounds__(sve::kThreads) init_rows_kernel(DevParams P, DevState<T> S, DevScalars* sc,
                                                                  double* mpart, long long k0, long long k1,
                                                                  unsigned b0, unsigned nb_total) {
  __shared__ double sh[2 * (sve::kThreads / 32)];
  __shared__ bool last;
  const long long k = k0 + (long long)blockIdx.x * sve::kThreads + threadIdx.x;
  double mh = 0.0, mz = 0.0;
  if (k < k1) {
    const int j = (int)(k / P.nx);
    const int i = (int)(k - (long long)j * P.nx);
    const long long e = sve::ext_index(P, i, j);
    T s[4] = {S.h[e], S.hu[e], P.dim == 2 ? S.hv[e] : T(0), S.z[e]};
    if (!(sve::tfinite(s[0]) && sve::tfinite(s[1]) && sve::tfinite(s[2]) && sve::tfinite(s[3])))
      atomicOr(&sc->status, sve::ST_NAN);
    else if (!sve::positive(s[0])) atomicOr(&sc->status, sve::ST_NEG_DEPTH);
    sve::store_cell(P, S, e, s, sve::tdiv(T(1), s[0]));
    sve::write_ghosts(P, S, i, j, s);
    mh = (double)s[0];
    mz = (double)s[3];
  }
  sve::block_sum2<sve::kThreads>(mh, mz, sh);
  if (threadIdx.x == 0) {
    mpart[2 * (b0 + blockIdx.x)] = mh;
    mpart[2 * (b0 + blockIdx.x) + 1] = mz;
    __threadfence();
    last = atomicAdd(&sc->done_cell, 1u) == nb_total - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  sc->mass_parts = nb_total;
  sc->done_cell = 0u;
}

// Host upload of the interior state in bands of rows on the upload stream,
// each band projected on the handle's stream as soon as it has arrived.
int upload_in_bands(sve_handle* h, const void* const src[4], int nbands) {
  const DevParams& P = step_params(h);
  const size_t row = h->elem * (size_t)P.nx, pitch = h->elem * (size_t)P.ex;
  SVE_TRY(cudaMemsetAsync(h->sc, 0, sizeof(DevScalars), h->stream));
  SVE_TRY(cudaEventRecord(h->up_ev[0], h->stream));  // the state may still be in use
  SVE_TRY(cudaStreamWaitEvent(h->upload, h->up_ev[0], 0));
  unsigned nb_total = 0;
  for (int c = 0; c < nbands; ++c) {
    const long long r0 = (long long)P.ny * c / nbands, r1 = (long long)P.ny * (c + 1) / nbands;
    nb_total += (unsigned)(((r1 - r0) * P.nx + sve::kThreads - 1) / sve::kThreads);
  }
  unsigned b0 = 0;
  for (int c = 0; c < nbands; ++c) {
    const long long r0 = (long long)P.ny * c / nbands, r1 = (long long)P.ny * (c + 1) / nbands;
    for (int f = 0; f < 4; ++f) {
      char* dst = (char*)h->fields[f] + h->elem * (size_t)(P.ex * (r0 + 1) + 1);
      const char* from = (const char*)src[f] + row * (size_t)r0;
      SVE_TRY(cudaMemcpy2DAsync(dst, pitch, from, row, row, (size_t)(r1 - r0), cudaMemcpyHostToDevice, h->upload));
    }
    SVE_TRY(cudaEventRecord(h->up_ev[1 + c], h->upload));
    SVE_TRY(cudaStreamWaitEvent(h->stream, h->up_ev[1 + c], 0));
    const unsigned nb = (unsigned)(((r1 - r0) * P.nx + sve::kThreads - 1) / sve::kThreads);
    if (h->cfg.precision == SVE_FP64)
      init_rows_kernel<double><<<nb, sve::kThreads, 0, h->stream>>>(P, state_of<double>(h), h->sc, h->mpart,
                                                                     r0 * P.nx, r1 * P.nx, b0, nb_total);
    else
      init_rows_kernel<float><<<nb, sve::kThreads, 0, h->stream>>>(P, state_of<float>(h), h->sc, h->mpart,
                                                                    r0 * P.nx, r1 * P.nx, b0, nb_total);
    b0 += nb;
  }
  return cudaGetLastError() == cudaSuccess ? SVE_OK : SVE_ERR_CUDA;
}

int run_steps(sve_handle* h, int nsteps, int fixed) {
  int rc = enqueue_steps(h, nsteps, fixed);
  if (rc) return rc;
  return wait_status(h);
}

// Upload, projection, checks and ghosts of a caller's state, enqueued on the
// handle's stream (status bits latched in the scalars, not read).
int enqueue_set_state(sve_handle* h, const void* depth, const void* hu, const void* hv, const void* zb, int where);
void* direct_ptr(void* p, int where);

}  // namespace

// Shared with sve_noalloc.cu and sve_adjoint.cu (not part of the C ABI).
__attribute__((visibility("hidden"))) int sve_internal_validate(const sve_config* c) { return validate(c); }
__attribute__((visibility("hidden"))) int sve_internal_reserve_dtlog(sve_handle* h, int n) {
  double* old = h->dtlog;
  const int rc = ensure_capacity(&h->dtlog, &h->dtlog_cap, n > 0 ? n : 1);
  if (h->dtlog != old) drop_graphs(h);  // graphs hold the dtlog pointer
  return rc;
}
__attribute__((visibility("hidden"))) void sve_internal_make_params(const sve_config* c, DevParams* P) {
  make_params(c, P);
}
__attribute__((visibility("hidden"))) int sve_internal_status_code(int st) { return status_to_code(st); }
// Whether a side of the configuration takes its ghost ring from outside (a
// block of a decomposed grid): only the handle's block calls can fill it.
__attribute__((visibility("hidden"))) bool sve_internal_has_external(const sve_config* c) {
  const int nsides = c->dim == 2 ? 4 : 2;
  for (int s = 0; s < nsides; ++s)
    if (c->bc[s] == SVE_BC_EXTERNAL) return true;
  return false;
}

extern "C" {

int sve_config_default(sve_config* c) {
  if (!c) return SVE_ERR_ARG;
  memset(c, 0, sizeof(*c));
  c->dim = 2;
  c->nx = 0;
  c->ny = 0;
  c->lx = 1.0;
  c->ly = 1.0;
  c->g = 9.81;
  c->cfl = 0.9;
  c->precision = SVE_FP64;
  c->bedload = SVE_GRASS;
  c->A_g = 1e-3;
  c->m_g = 3.0;
  c->s = 2.65;
  c->d_s = 1e-3;
  c->tau_cr = 0.05;
  c->friction = SVE_FRIC_NONE;
  c->bc[0] = SVE_BC_PERIODIC;
  c->bc[1] = SVE_BC_PERIODIC;
  c->bc[2] = SVE_BC_FREE;
  c->bc[3] = SVE_BC_FREE;
  c->kappa_a = 1.1;
  c->beta_min = 0.01;
  c->gamma_z = 2.0;
  c->newton_tol = 1e-9;
  c->newton_maxit = 30;
  return SVE_OK;
}

int sve_create(const sve_config* cfg, sve_handle** out) {
  if (!out) return SVE_ERR_ARG;
  *out = nullptr;
  int rc = validate(cfg);
  if (rc) return rc;
  sve_handle* h = new sve_handle();
  h->cfg = *cfg;
  make_params(cfg, &h->P);
  if (cudaGetDevice(&h->device) != cudaSuccess) { delete h; return SVE_ERR_CUDA; }
  h->elem = cfg->precision == SVE_FP64 ? 8 : 4;
  h->P_sw = h->P;  // the splitting scheme's shallow-water step: no transport
  h->P_sw.bedload = 0;
  h->P_sw.A_g = 0.0;
  h->P_sw.f.A_g = 0.0f;
  h->P_sw.m_g = 3.0;
  h->P_sw.f.m_g = 3.0f;
  h->P_sw.m_int = 3;
  h->next = (long long)(h->P.nx + 2) * (h->P.ny + 2);
  // block size of the two-kernel step: 128 threads, or one warp per block
  // while the grid is too small to give every SM two 256-thread blocks
  // (GB300 issues ~2 FP64 operations per clock per SM, so a small grid's FP64
  // work has to spread over many SMs)
  {
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) nsm = 152;
    h->nsm = nsm;
  }
  h->nt = auto_block_size(h);
  bool ok = true;
  for (int k = 0; k < 13 && ok; ++k) ok = cudaMalloc(&h->fields[k], h->elem * (size_t)h->next) == cudaSuccess;
  ok = ok && cudaMalloc(&h->fx, 8 * h->elem * (size_t)h->P.nfx) == cudaSuccess;
  ok = ok && cudaMalloc(&h->fy, 8 * h->elem * (size_t)(h->P.nfy > 0 ? h->P.nfy : 1)) == cudaSuccess;
  h->fused = cfg->precision == SVE_FP32 && cfg->dim == 2;
  // the carried update needs every ghost from a boundary rule (a block's
  // external ghosts are set by the caller between single steps)
  h->carry = h->fused;
  for (int k = 0; k < 4; ++k) h->carry = h->carry && cfg->bc[k] != SVE_BC_EXTERNAL;
  // its second state buffer: the projection planes tau, u, v, pi, which the
  // FP32 2D step does not read (the state upload fills them; no step reads
  // what the upload left there)
  if (h->carry)
    for (int k = 0; k < 4; ++k) h->alt[k] = h->fields[4 + k];
  if (h->fused) {
    h->march = sve::march_shape(h->P, h->nsm);
    h->agx = (h->P.nx + sve::kAThreads - 1) / sve::kAThreads;
    h->agy = std::min(h->P.ny, std::max(1, (h->nsm * (2048 / sve::kAThreads) + h->agx - 1) / h->agx));
  }
  // persistent small-grid step: one-warp blocks covering the larger of the
  // interface and cell counts, if that many are co-resident
  if (!h->fused) {
    const long long units = std::max((long long)h->P.nfx + h->P.nfy, (long long)h->P.nx * h->P.ny);
    const long long want = (units + sve::kPersistThreads - 1) / sve::kPersistThreads;
    int bs = 0;
    const cudaError_t oe =
        cfg->precision == SVE_FP64
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bs, sve::persistent_kernel<double>, sve::kPersistThreads, 0)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bs, sve::persistent_kernel<float>, sve::kPersistThreads, 0);
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device);
    h->pmax = (int)std::min<long long>((long long)bs * h->nsm, 4LL * h->nsm);
    if (oe == cudaSuccess && coop && bs > 0 && want <= h->pmax) {
      h->persist_ok = true;
      h->pgrid = (int)want;
    }
    cudaGetLastError();
  }
  const size_t nmp = std::max({2 * (size_t)sve::cell_blocks(h->P, sve::kThreadsNarrow),
                               2 * (size_t)std::max(1, h->agx * h->agy), 2 * (size_t)std::max(1, h->pmax)});
  ok = ok && cudaMalloc(&h->mpart, sizeof(double) * nmp) == cudaSuccess;
  ok = ok && cudaMalloc(&h->sc, sizeof(DevScalars)) == cudaSuccess;
  ok = ok && cudaMalloc(&h->ps, sizeof(sve::PersistScratch)) == cudaSuccess;
  if (!ok) { sve_destroy(h); return SVE_ERR_OOM; }
  if (ensure_capacity(&h->dtlog, &h->dtlog_cap, 1024)) { sve_destroy(h); return SVE_ERR_OOM; }
  if (ensure_capacity(&h->fixed, &h->fixed_cap, 1024)) { sve_destroy(h); return SVE_ERR_OOM; }
  if (cudaStreamCreateWithFlags(&h->capture, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->upload, cudaStreamNonBlocking) != cudaSuccess) {
    sve_destroy(h);
    return SVE_ERR_CUDA;
  }
  for (auto& e : h->up_ev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) { sve_destroy(h); return SVE_ERR_CUDA; }
  for (int k = 0; k < 13; ++k) cudaMemset(h->fields[k], 0, h->elem * (size_t)h->next);
  cudaMemset(h->sc, 0, sizeof(DevScalars));
  if (cudaDeviceSynchronize() != cudaSuccess) { sve_destroy(h); return SVE_ERR_CUDA; }
  *out = h;
  return SVE_OK;
}

int sve_set_stream(sve_handle* h, void* stream) {
  if (!h) return SVE_ERR_ARG;
  h->stream = (cudaStream_t)stream;
  return SVE_OK;
}

int sve_set_state(sve_handle* h, const void* depth, const void* hu, const void* hv, const void* zb, int where) {
  const int rc = enqueue_set_state(h, depth, hu, hv, zb, where);
  if (rc) return rc;
  DevScalars s;
  SVE_TRY(cudaMemcpyAsync(&s, h->sc, sizeof(s), cudaMemcpyDeviceToHost, h->stream));
  SVE_TRY(cudaStreamSynchronize(h->stream));
  return status_to_code(s.status);
}

int sve_advance(sve_handle* h, int nsteps, const void* depth_in, const void* hu_in, const void* hv_in,
                const void* zb_in, void* depth_out, void* hu_out, void* hv_out, void* zb_out, int where,
                double* t_out) {
  if (!h || nsteps < 1) return SVE_ERR_ARG;
  if (!depth_out || !hu_out || !zb_out || (h->cfg.dim == 2 && !hv_out)) return SVE_ERR_ARG;
  int rc = enqueue_set_state(h, depth_in, hu_in, hv_in, zb_in, where);
  if (rc) return rc;
  void* out[4] = {depth_out, hu_out, h->cfg.dim == 2 ? hv_out : nullptr, zb_out};
  const void* mirror[4] = {nullptr, nullptr, nullptr, nullptr};
  // Direct stores from the last cell update: into device memory always; into
  // page-locked host memory when that update is the FP64-bound cell kernel,
  // whose run time covers the host-link time of its stores.  The FP32 fused
  // step's apply pass is memory-bound, and host stores from it make it
  // link-bound (slower than a copy after it).
  bool direct = (where == SVE_DEVICE || !h->fused) && !h->scheme;  // (the split step's bed changes after the cell update)
  for (int f = 0; f < 4; ++f) {
    if (!out[f]) continue;
    mirror[f] = direct_ptr(out[f], where);
    direct = direct && mirror[f];
  }
  rc = enqueue_steps(h, nsteps, 0, direct ? mirror : nullptr);
  if (rc) return rc;
  if (!direct) {
    const DevParams& P = h->P;
    const size_t row = h->elem * (size_t)P.nx, pitch = h->elem * (size_t)P.ex;
    for (int f = 0; f < 4; ++f) {
      if (!out[f]) continue;
      const char* src = (const char*)h->fields[f] + h->elem * (size_t)(P.ex + 1);
      SVE_TRY(cudaMemcpy2DAsync(out[f], row, src, pitch, row, P.ny, cudaMemcpyDefault, h->stream));
    }
  }
  rc = wait_status(h);
  if (t_out && rc != SVE_ERR_CUDA) *t_out = h->last_t;
  return rc;
}

}  // extern "C"

namespace {

int enqueue_set_state(sve_handle* h, const void* depth, const void* hu, const void* hv, const void* zb, int where) {
  if (!h || !depth || !hu || !zb || (h->cfg.dim == 2 && !hv)) return SVE_ERR_ARG;
  if (where != SVE_HOST && where != SVE_DEVICE) return SVE_ERR_ARG;
  const DevParams& P = step_params(h);
  const size_t row = h->elem * (size_t)P.nx;
  const size_t pitch = h->elem * (size_t)P.ex;
  const cudaMemcpyKind kind = where == SVE_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const void* src[4] = {depth, hu, h->cfg.dim == 2 ? hv : nullptr, zb};
  // large 2D grids from the host: four bands of rows, each projected while
  // the next one is still arriving
  const int nbands = (where == SVE_HOST && h->cfg.dim == 2 && P.ny >= 64 && (long long)P.nx * P.ny >= (1LL << 18)) ? 4 : 1;
  if (nbands > 1) {
    const int urc = upload_in_bands(h, src, nbands);
    if (urc) return urc;
  } else {
    for (int f = 0; f < 4; ++f) {
      char* dst = (char*)h->fields[f] + h->elem * (size_t)(P.ex + 1);
      if (src[f]) SVE_TRY(cudaMemcpy2DAsync(dst, pitch, src[f], row, row, P.ny, kind, h->stream));
      else SVE_TRY(cudaMemsetAsync(h->fields[f], 0, h->elem * (size_t)h->next, h->stream));
    }
    SVE_TRY(cudaMemsetAsync(h->sc, 0, sizeof(DevScalars), h->stream));
    if (h->cfg.precision == SVE_FP64)
      sve::init_kernel<double><<<(unsigned)sve::cell_blocks(h->P, sve::kThreads), sve::kThreads, 0, h->stream>>>(P, state_of<double>(h), h->sc, h->mpart);
    else
      sve::init_kernel<float><<<(unsigned)sve::cell_blocks(h->P, sve::kThreads), sve::kThreads, 0, h->stream>>>(P, state_of<float>(h), h->sc, h->mpart);
  }
  SVE_TRY(cudaGetLastError());
  h->has_state = true;
  h->last_steps = 0;
  return SVE_OK;
}

// Device-accessible address of a caller's output buffer for direct stores
// from the kernels: device memory as it is, page-locked host memory through
// its device mapping; null for pageable host memory (copied instead).
void* direct_ptr(void* p, int where) {
  if (where == SVE_DEVICE) return p;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return (a.type == cudaMemoryTypeHost && a.devicePointer) ? a.devicePointer : nullptr;
}

}  // namespace

extern "C" {

int sve_step(sve_handle* h, int nsteps, double* t_out) {
  if (!h || nsteps < 0) return SVE_ERR_ARG;
  int rc = run_steps(h, nsteps, 0);
  if (t_out && rc != SVE_ERR_CUDA) *t_out = h->last_t;  // read back with the status
  return rc;
}

int sve_step_dt(sve_handle* h, int nsteps, const double* dts) {
  if (!h || nsteps < 0 || (nsteps > 0 && !dts)) return SVE_ERR_ARG;
  for (int k = 0; k < nsteps; ++k)
    if (!(dts[k] > 0.0) || !isfinite(dts[k])) return SVE_ERR_ARG;
  double* old = h->fixed;
  int rc = ensure_capacity(&h->fixed, &h->fixed_cap, nsteps > 0 ? nsteps : 1);
  if (rc) return rc;
  if (h->fixed != old) drop_graphs(h);
  if (nsteps > 0)
    SVE_TRY(cudaMemcpyAsync(h->fixed, dts, sizeof(double) * (size_t)nsteps, cudaMemcpyHostToDevice, h->stream));
  return run_steps(h, nsteps, 1);
}

int sve_get_state(sve_handle* h, void* depth, void* hu, void* hv, void* zb, int where) {
  if (!h) return SVE_ERR_ARG;
  if (!h->has_state) return SVE_ERR_STATE;
  if (where != SVE_HOST && where != SVE_DEVICE) return SVE_ERR_ARG;
  const DevParams& P = h->P;
  const size_t row = h->elem * (size_t)P.nx;
  const size_t pitch = h->elem * (size_t)P.ex;
  const cudaMemcpyKind kind = where == SVE_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  void* dst[4] = {depth, hu, hv, zb};
  for (int f = 0; f < 4; ++f) {
    if (!dst[f] || (f == 2 && h->cfg.dim == 1)) continue;
    const char* src = (const char*)h->fields[f] + h->elem * (size_t)(P.ex + 1);
    SVE_TRY(cudaMemcpy2DAsync(dst[f], row, src, pitch, row, P.ny, kind, h->stream));
  }
  SVE_TRY(cudaStreamSynchronize(h->stream));
  return SVE_OK;
}

int sve_get_diag(sve_handle* h, double* mass_h, double* mass_z, double* t, double* last_dt) {
  if (!h) return SVE_ERR_ARG;
  if (!h->has_state) return SVE_ERR_STATE;
  // the mass sums of the last step, from its per-block partials
  mass_kernel<<<1, sve::kThreads, 0, h->stream>>>(h->P, h->sc, h->mpart);
  SVE_TRY(cudaGetLastError());
  DevScalars s;
  SVE_TRY(cudaMemcpyAsync(&s, h->sc, sizeof(s), cudaMemcpyDeviceToHost, h->stream));
  SVE_TRY(cudaStreamSynchronize(h->stream));
  if (mass_h) *mass_h = s.mass_h;
  if (mass_z) *mass_z = s.mass_z;
  if (t) *t = s.t;
  if (last_dt) *last_dt = s.dt;
  return status_to_code(s.status);
}

int sve_get_dts(sve_handle* h, double* dts, int n) {
  if (!h || n < 0 || (n > 0 && !dts)) return SVE_ERR_ARG;
  int m = n < h->last_steps ? n : h->last_steps;
  if (m > 0) {
    SVE_TRY(cudaMemcpyAsync(dts, h->dtlog, sizeof(double) * (size_t)m, cudaMemcpyDeviceToHost, h->stream));
    SVE_TRY(cudaStreamSynchronize(h->stream));
  }
  return m;
}

void sve_destroy(sve_handle* h) {
  if (!h) return;
  sve_internal_adjoint_free(h);
  drop_graphs(h);
  cudaStreamSynchronize(h->stream);
  for (auto e : h->events) cudaEventDestroy(e);
  for (auto& f : h->fields)
    if (f) cudaFree(f);
  if (h->fx) cudaFree(h->fx);
  if (h->fy) cudaFree(h->fy);
  if (h->zsave) cudaFree(h->zsave);
  if (h->hist) cudaFree(h->hist);
  if (h->mpart) cudaFree(h->mpart);
  if (h->sc) cudaFree(h->sc);
  if (h->ps) cudaFree(h->ps);
  if (h->halo) cudaFree(h->halo);
  if (h->dtlog) cudaFree(h->dtlog);
  if (h->fixed) cudaFree(h->fixed);
  if (h->capture) cudaStreamDestroy(h->capture);
  if (h->upload) cudaStreamDestroy(h->upload);
  for (auto& e : h->up_ev)
    if (e) cudaEventDestroy(e);
  delete h;
}

const char* sve_strerror(int code) {
  switch (code) {
    case SVE_OK: return "ok";
    case SVE_ERR_ARG: return "invalid argument";
    case SVE_ERR_CUDA: return "CUDA runtime error";
    case SVE_ERR_OOM: return "out of device memory";
    case SVE_ERR_NEG_DEPTH: return "non-positive water depth";
    case SVE_ERR_RIEMANN: return "Riemann problem without a solution with positive specific volumes";
    case SVE_ERR_NAN: return "non-finite value in the state";
    case SVE_ERR_DT: return "invalid time step";
    case SVE_ERR_STATE: return "no state set";
    case SVE_ERR_NOALLOC_SIZE: return "grid too large for the static scratch of sve_step_noalloc";
    case SVE_ERR_SYNC: return "a grid-wide wait of the persistent step ran out";
    default: return "unknown error";
  }
}

int sve_set_block_size(sve_handle* h, int threads) {
  if (!h) return SVE_ERR_ARG;
  if (threads != 0 && threads != sve::kThreadsNarrow && threads != sve::kThreadsStep && threads != sve::kThreads)
    return SVE_ERR_ARG;
  const int nt = threads == 0 ? auto_block_size(h) : threads;
  if (nt != h->nt) drop_graphs(h);  // the captured steps hold the launch shape
  h->nt = nt;
  return SVE_OK;
}

int sve_get_block_size(sve_handle* h) {
  if (!h) return SVE_ERR_ARG;
  return h->nt;
}

int sve_set_persistent(sve_handle* h, int on) {
  if (!h || on < 0 || on > 1) return SVE_ERR_ARG;
  h->persist_mode = on;
  return SVE_OK;
}

int sve_get_persistent(sve_handle* h) {
  if (!h) return SVE_ERR_ARG;
  return use_persistent(h) ? 1 : 0;
}

int sve_set_scheme(sve_handle* h, int scheme) {
  if (!h || (scheme != SVE_SCHEME_COUPLED && scheme != SVE_SCHEME_SPLIT)) return SVE_ERR_ARG;
  if (scheme == SVE_SCHEME_SPLIT && (h->cfg.precision != SVE_FP64 || sve_internal_has_external(&h->cfg)))
    return SVE_ERR_ARG;
  if (scheme == h->scheme) return SVE_OK;
  if (scheme == SVE_SCHEME_SPLIT && !h->zsave &&
      cudaMalloc(&h->zsave, sizeof(double) * (size_t)h->next) != cudaSuccess)
    return SVE_ERR_OOM;
  drop_graphs(h);  // they hold the other step
  h->scheme = scheme;
  if (!h->has_state) return SVE_OK;
  // the current state projected for the new step's parameters
  sve::init_kernel<double><<<(unsigned)sve::cell_blocks(h->P, sve::kThreads), sve::kThreads, 0, h->stream>>>(
      step_params(h), state_of<double>(h), h->sc, h->mpart);
  return wait_status(h);
}

int sve_get_scheme(sve_handle* h) { return h ? h->scheme : SVE_ERR_ARG; }

int sve_set_history(sve_handle* h, int capacity) {
  if (!h || capacity < 0) return SVE_ERR_ARG;
  if (capacity != h->hist_cap) {
    SVE_TRY(cudaStreamSynchronize(h->stream));
    if (h->hist) cudaFree(h->hist);
    h->hist = nullptr;
    h->hist_cap = 0;
    if (capacity > 0 && cudaMalloc(&h->hist, sizeof(double) * 6 * (size_t)capacity) != cudaSuccess) return SVE_ERR_OOM;
    h->hist_cap = capacity;
    drop_graphs(h);  // they hold the step without (or with) its record
  }
  SVE_TRY(cudaMemsetAsync(&h->sc->hist_count, 0, sizeof(unsigned long long), h->stream));
  return SVE_OK;
}

int sve_get_history(sve_handle* h, double* records, int n) {
  if (!h || n < 0 || (n > 0 && !records)) return SVE_ERR_ARG;
  if (h->hist_cap == 0) return SVE_ERR_STATE;
  unsigned long long count = 0;
  SVE_TRY(cudaMemcpyAsync(&count, &h->sc->hist_count, sizeof(count), cudaMemcpyDeviceToHost, h->stream));
  SVE_TRY(cudaStreamSynchronize(h->stream));
  const unsigned long long avail = count < (unsigned long long)h->hist_cap ? count : (unsigned long long)h->hist_cap;
  const int m = (int)(avail < (unsigned long long)n ? avail : (unsigned long long)n);
  // the last m records, oldest first: at most two pieces of the ring
  const size_t start = (size_t)((count - (unsigned long long)m) % (unsigned long long)h->hist_cap);
  const size_t first = std::min((size_t)m, (size_t)h->hist_cap - start);
  if (first > 0)
    SVE_TRY(cudaMemcpyAsync(records, h->hist + 6 * start, sizeof(double) * 6 * first, cudaMemcpyDeviceToHost,
                            h->stream));
  if ((size_t)m > first)
    SVE_TRY(cudaMemcpyAsync(records + 6 * first, h->hist, sizeof(double) * 6 * ((size_t)m - first),
                            cudaMemcpyDeviceToHost, h->stream));
  SVE_TRY(cudaStreamSynchronize(h->stream));
  return m;
}

int sve_check_sync_timeout(sve_handle* h, long long polls) {
  if (!h || polls < 1) return SVE_ERR_ARG;
  if (!h->has_state) return SVE_ERR_STATE;
  if (!h->persist_ok) return SVE_ERR_ARG;
  SVE_TRY(cudaMemsetAsync(&h->sc->call_step, 0, sizeof(int), h->stream));
  // one arrival more than there are blocks: the first barrier never opens
  const int rc = launch_persistent(h, 1, 0, (unsigned int)h->pgrid + 1u, polls);
  if (rc) return rc;
  h->last_launches = 1;
  h->last_steps = 0;
  return wait_status(h);
}

long long sve_last_launch_count(sve_handle* h) { return h ? h->last_launches : -1; }

int sve_step_async(sve_handle* h, int nsteps) {
  if (!h || nsteps < 0) return SVE_ERR_ARG;
  return enqueue_steps(h, nsteps, 0);
}

int sve_sync(sve_handle* h) {
  if (!h) return SVE_ERR_ARG;
  if (!h->has_state) return SVE_ERR_STATE;
  return wait_status(h);
}

int sve_profile(sve_handle* h, int on) {
  if (!h) return SVE_ERR_ARG;
  int rc = drain_events(h);
  h->profiling = on != 0;
  h->prof_ms[0] = h->prof_ms[1] = 0.0;
  h->prof_launches[0] = h->prof_launches[1] = 0;
  return rc;
}

int sve_profile_read(sve_handle* h, double* ms, long long* launches) {
  if (!h || !ms || !launches) return SVE_ERR_ARG;
  int rc = drain_events(h);
  if (rc) return rc;
  ms[0] = h->prof_ms[0];
  ms[1] = h->prof_ms[1];
  launches[0] = h->prof_launches[0];
  launches[1] = h->prof_launches[1];
  return SVE_OK;
}

int sve_get_counters(sve_handle* h, long long* steps, unsigned long long* newton_iters) {
  if (!h) return SVE_ERR_ARG;
  if (!h->has_state) return SVE_ERR_STATE;
  DevScalars s;
  SVE_TRY(cudaMemcpyAsync(&s, h->sc, sizeof(s), cudaMemcpyDeviceToHost, h->stream));
  SVE_TRY(cudaStreamSynchronize(h->stream));
  if (steps) *steps = s.steps;
  if (newton_iters) *newton_iters = s.newton_iters;
  return status_to_code(s.status);
}

int sve_get_safeguards(sve_handle* h, unsigned long long* halvings, unsigned long long* raised,
                       unsigned long long* retries) {
  if (!h) return SVE_ERR_ARG;
  if (!h->has_state) return SVE_ERR_STATE;
  DevScalars s;
  SVE_TRY(cudaMemcpyAsync(&s, h->sc, sizeof(s), cudaMemcpyDeviceToHost, h->stream));
  SVE_TRY(cudaStreamSynchronize(h->stream));
  if (halvings) *halvings = s.halvings;
  if (raised) *raised = s.raised;
  if (retries) *retries = s.retries;
  return status_to_code(s.status);
}

}  // extern "C"
