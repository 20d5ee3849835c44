// sve_adjoint.cu -- hand-written discrete adjoint of the step (include/sve.h,
// sve_record_forward / sve_adjoint).
//
// Step n maps U^n to U^{n+1} = Fric(U^n - dt_n/dx (A+ + A-) - dt_n/dy (...))
// with the time steps dt_n recorded by the forward run and held fixed.  The
// reverse sweep propagates lambda^n = (dU^{n+1}/dU^n)^T lambda^{n+1}:
//   adj_friction_kernel  mu = (dFric/dU~)^T lambda^{n+1} per cell (closed form),
//                        and the friction coefficient's gradient;
//   adj_cells_kernel     the projection of every cell (ghosts included) with
//                        the record its backward sweep needs, once per step;
//   adj_interface_kernel per interface, the product of the transposed
//                        Jacobian of (A-, A+) -- with respect to both cells'
//                        conserved states, A_g and m_g -- with mu of both
//                        cells, in reverse mode (interface_vjp_cells of
//                        sve_adjoint_jac.cuh: one value pass through the
//                        step's own templates at the kept Newton root, one
//                        hand-written backward sweep; the root enters through
//                        the implicit function theorem), up to the transport
//                        law: the cotangents of the cells' Omega and dQ are
//                        passed on; tested against forward-mode dual numbers
//                        through the same templates;
//   adj_gather_kernel    lambda^n = mu + the contributions of the cell's four
//                        interfaces, the law's part of the cell's projection
//                        once per frame for the sum of its two interfaces, ghost
//                        cells routed back to the cells they copy (the
//                        transposed ghost rule); the law parameters' gradients.
// Forward states are recomputed per segment from checkpoints taken every C
// steps (C ~ sqrt(N)): memory of ~2 sqrt(N) states, one extra forward pass.
// Supported: FP64 state, Grass bedload (A_g, m_g), any friction law (its
// coefficient: K for Strickler, f for Darcy-Weisbach), every boundary rule.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <vector>

#include "../../include/sve.h"
#include "sve_device.cuh"
#include "sve_adjoint_jac.cuh"
#include "sve_handle.h"

using sve::Cell;
using sve::DevParams;
using sve::DevScalars;
using sve::DevState;
using sve::Dual;
using sve::NewtonConst;
using sve::NewtonEval;

struct sve_adjoint_rec {
  int nsteps = 0;
  int every = 0;
  int ncp = 0;                      // segments of `every` steps (the last one shorter)
  bool stored = false;              // every step's states kept by the recording (no recompute)
  // segments kept_from .. ncp - 1 (checkpoint mode): their steps' padded and
  // convected states, roots and doublings kept by the recording, so that the
  // reverse sweep recomputes only the earlier segments
  int kept_from = 0;
  double* kseg = nullptr;
  double* ksegc = nullptr;
  double* kroots = nullptr;
  unsigned char* krtry = nullptr;
  std::vector<double> dts;          // dt of each recorded step
  std::vector<double*> checkpoints;  // padded (h, hu, hv, z) at steps 0, C, 2C, ...
  double* seg = nullptr;            // padded states of one segment (C of them)
  size_t seg_cap = 0;
  double* segc = nullptr;           // their convected (pre-friction) interior states, 4 planes each
  size_t segc_cap = 0;
  double* roots = nullptr;          // their interfaces' Newton roots p* (x then y interfaces, one plane a step)
  size_t roots_cap = 0;
  unsigned char* rtry = nullptr;    // and the doublings of a of those solves
  size_t rtry_cap = 0;
  double* cells = nullptr;          // per-cell projection record of the state being reversed (adj_cells_kernel)
  size_t cells_cap = 0;
  double* q = nullptr;              // per interface, the cotangents of both cells' (Omega, dQ) (4 planes)
  size_t q_cap = 0;
  double* lam = nullptr;            // 2 x 4 interior planes (current, next)
  double* mu = nullptr;             // 4 interior planes
  double* gpart = nullptr;          // per-block parameter partials
  size_t gpart_cap = 0;
  double* gacc = nullptr;           // [3] accumulated parameter gradients + counters
  unsigned int* done = nullptr;
  double t0 = 0.0;
};

namespace {

constexpr int kAdjThreads = 128;

// Deterministic sum of per-block partials (nper <= 2 per block) into
// acc[0..nper-1] by the last block of the launch: thread t adds blocks t,
// t + NT, ... in order (L2 loads, several in flight), then a fixed tree.
template <int NT>
__device__ __forceinline__ void finish_partials(const double* part, int nper, double* acc, unsigned int* done) {
  __shared__ bool last;
  __shared__ double sh[2 * (NT / 32)];
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s0 = 0.0, s1 = 0.0;
#pragma unroll 4
  for (unsigned b = threadIdx.x; b < gridDim.x; b += NT) {
    s0 += __ldcg(part + (size_t)nper * b);
    if (nper > 1) s1 += __ldcg(part + (size_t)nper * b + 1);
  }
  sve::block_sum2<NT>(s0, s1, sh);
  if (threadIdx.x == 0) {
    acc[0] += s0;
    if (nper > 1) acc[1] += s1;
    *done = 0u;
  }
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kAdjThreads / 32; ++w) r += sh[w];
  __syncthreads();
  return r;
}

// The convected (pre-friction) state U~ of every interior cell for the step
// whose fluctuations the planes of S hold (4 planes of nx ny) and whose time
// step the interface pass left in sc->dt, kept for the friction adjoint.
__global__ void __launch_bounds__(kAdjThreads) convect_save_kernel(DevParams P, DevState<double> S,
                                                                   const DevScalars* sc, double* out) {
  const long long ncell = (long long)P.nx * P.ny;
  const long long k = (long long)blockIdx.x * kAdjThreads + threadIdx.x;
  if (k >= ncell) return;
  const double dt = sc->dt;
  const int j = (int)(k / P.nx), i = (int)(k - (long long)j * P.nx);
  double s[4];
  sve::convect_cell(P, S, i, j, sve::ext_index(P, i, j), dt, s);
#pragma unroll
  for (int f = 0; f < 4; ++f) out[f * ncell + k] = s[f];
}

// mu = (dFric/dU~)^T lambda^{n+1} per interior cell, U~ = conv (the saved
// convected state of the step); gradient of the friction coefficient.
// Fric: q <- q / den, den = 1 + dt C(h) |q|.
__global__ void __launch_bounds__(kAdjThreads) adj_friction_kernel(DevParams P, const double* conv,
                                                                   const double* lam, double* mu, double dt,
                                                                   double* gpart, double* gacc,
                                                                   unsigned int* done) {
  __shared__ double sh[kAdjThreads / 32];
  const long long ncell = (long long)P.nx * P.ny;
  const long long k = (long long)blockIdx.x * kAdjThreads + threadIdx.x;
  double gk = 0.0;
  if (k < ncell) {
    const double s[4] = {conv[k], conv[ncell + k], conv[2 * ncell + k], conv[3 * ncell + k]};
    const double lh = lam[k], l1 = lam[ncell + k], l2 = lam[2 * ncell + k], lz = lam[3 * ncell + k];
    double mh = lh, m1 = l1, m2 = l2;
    if (P.friction != 0) {
      // C(h) and den as the step's friction computes them; one divide for
      // 1/den and 1/|q|
      const double h = s[0], q1 = s[1], q2 = s[2];
      const double qn = sqrt(fma(q1, q1, q2 * q2));
      const double tau = 1.0 / h;
      double C = P.fric_c * (tau * tau);
      if (P.friction == 2) C = C * sve::rcbrt64(h);
      const double den = 1.0 + dt * C * qn;
      double id, iqn = 0.0;
      if (qn > 0.0) {
        const double r = 1.0 / (den * qn);
        id = r * qn;
        iqn = r * den;
      } else {
        id = 1.0 / den;
      }
      const double id2 = id * id;
      // dC/dh = -2 C / h (Darcy), -7/3 C / h (Strickler)
      const double dCdh = (P.friction == 1 ? -2.0 : -7.0 / 3.0) * C * tau;
      const double lq = l1 * q1 + l2 * q2;  // lambda . q
      mh = lh - lq * dt * qn * dCdh * id2;
      if (qn > 0.0) {
        const double f = dt * C * iqn * id2;
        m1 = l1 * id - lq * f * q1;
        m2 = l2 * id - lq * f * q2;
      } else {
        m1 = l1 * id;
        m2 = l2 * id;
      }
      // coefficient: Strickler K (C = g / (K^2 h^(7/3)): dC/dK = -2 C / K);
      // Darcy f (C = f / (8 h^2): dC/df = C / f)
      const double dCdk = P.friction == 2 ? -2.0 * C / P.fric_coef : C / P.fric_coef;
      gk = -lq * dt * qn * dCdk * id2;
    }
    mu[k] = mh;
    mu[ncell + k] = m1;
    mu[2 * ncell + k] = m2;
    mu[3 * ncell + k] = lz;
  }
  const double b = block_sum(gk, sh);
  if (threadIdx.x == 0) gpart[blockIdx.x] = b;
  finish_partials<kAdjThreads>(gpart, 1, gacc + 2, done);
}

// Planes of the per-cell projection record (padded cells, plane k at
// cells + k * next): what the interface adjoint reads instead of projecting
// both its cells itself (each cell then projected once per step, not once
// per interface side).  Grass / Shields-parameter law:
enum AdjCellPlane {
  kCTau, kCPi, kCCa,
  kCSp,                // |U|            / s2 = |U|^2
  kCIsp,               // 1/|U| (0 where |U| = 0; Shields: 0 where no transport)
  kCLsp,               // log |U|        / alpha
  kCPm1,               // |U|^(m-1)      / q*
  kCPm3,               // |U|^(m-3)      / dq*/dtau*
  kCDdq,               // -              / d2q*/dtau*2
  kCU, kCV,            // velocities
  kCOmx, kCCbx, kCIcbx, kCDQx,  // x frame: Omega, cb, 1/cb, dQ/du
  kCOmy, kCCby, kCIcby, kCDQy,  // y frame
  kCPlanes
};

// The projection record of every padded cell with a positive depth, in the
// x frame and (2D) the y frame, by the adjoint's own projection
// (project_grass_rec / project_shields_rec in the x frame; in the y frame
// only Omega, dQ, cb and 1/cb differ).
template <bool GRASS>
__global__ void __launch_bounds__(kAdjThreads) adj_cells_kernel(DevParams P, DevState<double> S, double A,
                                                                double m, double* cells, long long next) {
  const long long e = (long long)blockIdx.x * kAdjThreads + threadIdx.x;
  if (e >= next) return;
  const double H = S.h[e], Hu = S.hu[e], Hv = P.dim == 2 ? S.hv[e] : 0.0, Z = S.z[e];
  if (!(H > 0.0)) return;  // corners of the padding: never an interface's cell
  auto put = [&](int k, double v) { cells[(long long)k * next + e] = v; };
  sve::ProjRec r;
  const Cell<double> cx = GRASS ? sve::project_grass_rec(P, H, Hu, Hv, Z, A, m, r)
                                : sve::project_shields_rec(P, H, Hu, Hv, Z, r);
  put(kCTau, cx.tau); put(kCPi, cx.Pi); put(kCCa, cx.ca);
  put(kCSp, GRASS ? r.sp : r.s2);
  put(kCIsp, r.isp);
  put(kCLsp, GRASS ? r.lsp : r.alpha);
  put(kCPm1, GRASS ? r.pm1 : r.q);
  put(kCPm3, GRASS ? r.pm3 : r.dq);
  put(kCDdq, GRASS ? 0.0 : r.ddq);
  put(kCU, cx.un); put(kCV, cx.ut);
  put(kCOmx, cx.Om); put(kCCbx, cx.cb); put(kCIcbx, r.icb); put(kCDQx, r.dQ);
  if (P.dim == 2) {
    // y frame: normal velocity v, tangential u
    double Q, dQ;
    if (GRASS) sve::grass_q(r, cx.ut, A, m, Q, dQ);
    else sve::shields_q(P, r, cx.ut, cx.un, Q, dQ);
    const double cb = sqrt(Hv * Hv + P.g * H * H * dQ);
    put(kCOmy, Q); put(kCCby, cb); put(kCIcby, cb > 0.0 ? 1.0 / cb : 0.0); put(kCDQy, dQ);
  }
}

// The projected cell at padded index e in the frame of an x (ydir false) or
// y interface, and its record, from the planes of adj_cells_kernel.
template <bool GRASS>
__device__ __forceinline__ Cell<double> adj_load_cell(const DevState<double>& S, const double* cells,
                                                      long long next, long long e, bool ydir, sve::ProjRec& r) {
  auto get = [&](int k) { return cells[(long long)k * next + e]; };
  Cell<double> c;
  c.H = S.h[e];
  c.Hn = ydir ? S.hv[e] : S.hu[e];
  c.Ht = ydir ? S.hu[e] : S.hv[e];
  c.Z = S.z[e];
  c.tau = get(kCTau);
  const double u = get(kCU), v = get(kCV);
  c.un = ydir ? v : u;
  c.ut = ydir ? u : v;
  c.Pi = get(kCPi);
  c.ca = get(kCCa);
  c.Om = get(ydir ? kCOmy : kCOmx);
  c.cb = get(ydir ? kCCby : kCCbx);
  r.H = c.H; r.Hn = c.Hn; r.Ht = c.Ht; r.tau = c.tau; r.un = c.un; r.ut = c.ut; r.ca = c.ca; r.cb = c.cb;
  r.icb = get(ydir ? kCIcby : kCIcbx);
  r.dQ = get(ydir ? kCDQy : kCDQx);
  r.isp = get(kCIsp);
  if (GRASS) {
    r.sp = get(kCSp);
    r.lsp = get(kCLsp);
    r.pm1 = get(kCPm1);
    r.pm3 = get(kCPm3);
    r.still = r.sp == 0.0;
  } else {
    r.s2 = get(kCSp);
    r.alpha = get(kCLsp);
    r.q = get(kCPm1);
    r.dq = get(kCPm3);
    r.ddq = get(kCDdq);
    r.active = r.isp > 0.0;
    r.still = r.s2 == 0.0;
    r.sp = 0.0;
    r.lsp = 0.0;
  }
  return c;
}

// Per interface: the Jacobian-transpose product of its fluctuations with mu of
// its two cells (a ghost side has mu = 0) up to the transport law: the
// cotangents of both cells' conserved states in the fluctuation planes (8
// values: left state then right state, interface frame) and those of both
// cells' (Omega, dQ) in the planes of q (4 values: left then right), which
// adj_gather_kernel takes through the law once per cell.  The cells'
// projections and records come from the planes of adj_cells_kernel.
template <bool GRASS>
__global__ void __launch_bounds__(kAdjThreads) adj_interface_kernel(DevParams P, DevState<double> S,
                                                                    const double* mu, double dt, double A,
                                                                    double m, const double* roots,
                                                                    const unsigned char* rtry, const double* cells,
                                                                    long long next, double* q) {
  const long long ncell = (long long)P.nx * P.ny;
  const long long nall = P.nfx + P.nfy;
  const long long idx = (long long)blockIdx.x * kAdjThreads + threadIdx.x;
  if (idx >= nall) return;
  const bool ydir = idx >= P.nfx;
  const long long k = ydir ? idx - P.nfx : idx;
  int iL, jL, iR, jR;
  if (!ydir) {
    jR = (int)(k / (P.nx + 1));
    iR = (int)(k - (long long)jR * (P.nx + 1));
    iL = iR - 1;
    jL = jR;
  } else {
    jR = (int)(k / P.nx);
    iR = (int)(k - (long long)jR * P.nx);
    iL = iR;
    jL = jR - 1;
  }
  const long long eL = sve::ext_index(P, iL, jL), eR = sve::ext_index(P, iR, jR);
  const bool inL = iL >= 0 && iL < P.nx && jL >= 0 && jL < P.ny;
  const bool inR = iR >= 0 && iR < P.nx && jR >= 0 && jR < P.ny;
  const int cn = ydir ? 2 : 1, ct = ydir ? 1 : 2;  // normal / tangential component in (h, hu, hv, z)
  double muL[4] = {0, 0, 0, 0}, muR[4] = {0, 0, 0, 0};
  if (inL) {
    const long long c = (long long)jL * P.nx + iL;
    muL[0] = mu[c]; muL[1] = mu[cn * ncell + c]; muL[2] = mu[ct * ncell + c]; muL[3] = mu[3 * ncell + c];
  }
  if (inR) {
    const long long c = (long long)jR * P.nx + iR;
    muR[0] = mu[c]; muR[1] = mu[cn * ncell + c]; muR[2] = mu[ct * ncell + c]; muR[3] = mu[3 * ncell + c];
  }
  double ub[8] = {0, 0, 0, 0, 0, 0, 0, 0}, qb[4] = {0, 0, 0, 0};
  bool any = false;
#pragma unroll
  for (int c = 0; c < 4; ++c) any = any || muL[c] != 0.0 || muR[c] != 0.0;
  if (any) {
    sve::ProjRec rL, rR;
    const Cell<double> L = adj_load_cell<GRASS>(S, cells, next, eL, ydir, rL);
    const Cell<double> R = adj_load_cell<GRASS>(S, cells, next, eR, ydir, rR);
    // reverse mode: the transposed Jacobian of the fluctuations applied
    // to -dt/dx (mu of the left cell, mu of the right cell)
    const double w = -dt * (ydir ? P.inv_dy : P.inv_dx);
    double Amb[4], Apb[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) { Amb[c] = w * muL[c]; Apb[c] = w * muR[c]; }
    double Ab = 0.0, mb = 0.0, Kb = 0.0;  // (the laws' part is adj_gather_kernel's)
    // (the forward run solved this interface at this state; a failure here
    // leaves its contribution at zero, as the value pass did before) the
    // forward solve's root (kept by the recording or the segment's
    // recompute) spares the value pass its Newton iteration
    sve::interface_vjp_cells<GRASS>(P, L, R, rL, rR, A, m, Amb, Apb, ub, Ab, mb, Kb, roots[idx], (int)rtry[idx],
                                    qb);
  }
  double* v = ydir ? S.fy : S.fx;
  const long long nf = ydir ? P.nfy : P.nfx;
#pragma unroll
  for (int c = 0; c < 8; ++c) v[c * nf + k] = ub[c];
#pragma unroll
  for (int c = 0; c < 4; ++c) q[c * nall + idx] = qb[c];
}

// Transposed ghost rule of side s in the side's frame (h, normal, tangential,
// z): periodic / free copy, inflow_q keeps h and z, inflow_qh keeps z, wall
// mirrors the normal discharge.
__device__ __forceinline__ void ghost_transpose(int type, double g[4]) {
  switch (type) {
    case sve::GHOST_INFLOW_Q: g[1] = 0.0; g[2] = 0.0; break;
    case sve::GHOST_INFLOW_QH: g[0] = 0.0; g[1] = 0.0; g[2] = 0.0; break;
    case sve::GHOST_WALL: g[1] = -g[1]; break;
    default: break;
  }
}

// The law's part of a cell's (or ghost's) projection backward in one frame:
// the cotangents (Qb, dQb) of its Omega and dQ, summed over the interfaces of
// that frame, taken to its conserved state (H, Hn, Ht) in the frame order.
template <bool GRASS>
__device__ __forceinline__ void law_bar(const DevParams& P, const DevState<double>& S, const double* cells,
                                        long long next, long long e, bool ydir, double A, double m, double Qb,
                                        double dQb, double g[3], double& Ab, double& mb, double& Kb) {
  if (Qb == 0.0 && dQb == 0.0) return;
  sve::ProjRec r;
  adj_load_cell<GRASS>(S, cells, next, e, ydir, r);
  double unb = 0.0, utb = 0.0, Hb = 0.0, Hnb = 0.0, Htb = 0.0;
  sve::closure_bar<GRASS>(P, r, A, m, Qb, dQb, unb, utb, Hb, Ab, mb, Kb);
  sve::vel_fold_bar(r, unb, utb, 0.0, Hb, Hnb, Htb);
  g[0] += Hb;
  g[1] += Hnb;
  g[2] += Htb;
}

// lambda^n per interior cell: mu, plus the cotangents of the cell's four
// interfaces (their conserved parts, and the law's part of the cell's
// projection for the sum over each frame's two interfaces), ghost cells
// routed back to the cells they copy (the law's part with the ghost's own
// record, then the transposed ghost rule); the parameters' gradients of the
// law's part accumulated.
template <bool GRASS>
__global__ void __launch_bounds__(kAdjThreads) adj_gather_kernel(DevParams P, DevState<double> S, const double* mu,
                                                                 const double* q, const double* cells,
                                                                 long long next, double A, double m, double* lam,
                                                                 double* gpart, double* gacc, unsigned int* done) {
  __shared__ double sh[kAdjThreads / 32];
  const long long ncell = (long long)P.nx * P.ny;
  const long long k = (long long)blockIdx.x * kAdjThreads + threadIdx.x;
  double Ab = 0.0, mb = 0.0, Kb = 0.0;
  if (k < ncell) {
    const int j = (int)(k / P.nx), i = (int)(k - (long long)j * P.nx);
    const long long nfx = P.nfx, nfy = P.nfy, nall = nfx + nfy;
    const long long e = sve::ext_index(P, i, j);
    double r[4] = {mu[k], mu[ncell + k], mu[2 * ncell + k], mu[3 * ncell + k]};
    // x: as the right cell of interface (i - 1/2, j), as the left cell of (i + 1/2, j)
    const long long kx = (long long)j * (P.nx + 1) + i;
#pragma unroll
    for (int c = 0; c < 4; ++c) r[c] += S.fx[(4 + c) * nfx + kx] + S.fx[c * nfx + kx + 1];
    {
      double g[3] = {0.0, 0.0, 0.0};
      law_bar<GRASS>(P, S, cells, next, e, false, A, m, q[2 * nall + kx] + q[kx + 1],
                     q[3 * nall + kx] + q[nall + kx + 1], g, Ab, mb, Kb);
      r[0] += g[0]; r[1] += g[1]; r[2] += g[2];
    }
    if (P.dim == 2) {
      // y frame (h, hv, hu, z)
      const long long ky = (long long)j * P.nx + i;
      const double* y = S.fy;
      r[0] += y[4 * nfy + ky] + y[0 * nfy + ky + P.nx];
      r[2] += y[5 * nfy + ky] + y[1 * nfy + ky + P.nx];
      r[1] += y[6 * nfy + ky] + y[2 * nfy + ky + P.nx];
      r[3] += y[7 * nfy + ky] + y[3 * nfy + ky + P.nx];
      double g[3] = {0.0, 0.0, 0.0};
      const long long qy = nfx + ky;
      law_bar<GRASS>(P, S, cells, next, e, true, A, m, q[2 * nall + qy] + q[qy + P.nx],
                     q[3 * nall + qy] + q[nall + qy + P.nx], g, Ab, mb, Kb);
      r[0] += g[0]; r[2] += g[1]; r[1] += g[2];
    }
    // ghosts this cell feeds: their adjoint flows back through the ghost rule
    double g[4];
    const bool perx = P.bc[0] == sve::GHOST_PERIODIC;
    if ((!perx && i == 0) || (perx && i == P.nx - 1)) {  // W ghost: left state of (0 - 1/2, j)
      const long long kk = (long long)j * (P.nx + 1);
      for (int c = 0; c < 4; ++c) g[c] = S.fx[c * nfx + kk];
      law_bar<GRASS>(P, S, cells, next, sve::ext_index(P, -1, j), false, A, m, q[kk], q[nall + kk], g, Ab, mb, Kb);
      ghost_transpose(P.bc[0], g);
      for (int c = 0; c < 4; ++c) r[c] += g[c];
    }
    if ((!perx && i == P.nx - 1) || (perx && i == 0)) {  // E ghost: right state of (nx - 1/2, j)
      const long long kk = (long long)j * (P.nx + 1) + P.nx;
      for (int c = 0; c < 4; ++c) g[c] = S.fx[(4 + c) * nfx + kk];
      law_bar<GRASS>(P, S, cells, next, sve::ext_index(P, P.nx, j), false, A, m, q[2 * nall + kk],
                     q[3 * nall + kk], g, Ab, mb, Kb);
      ghost_transpose(P.bc[1], g);
      for (int c = 0; c < 4; ++c) r[c] += g[c];
    }
    if (P.dim == 2) {
      const bool pery = P.bc[2] == sve::GHOST_PERIODIC;
      if ((!pery && j == 0) || (pery && j == P.ny - 1)) {  // S ghost: left state of (i, 0 - 1/2)
        const long long kk = i;
        for (int c = 0; c < 4; ++c) g[c] = S.fy[c * nfy + kk];
        law_bar<GRASS>(P, S, cells, next, sve::ext_index(P, i, -1), true, A, m, q[nfx + kk], q[nall + nfx + kk], g,
                       Ab, mb, Kb);
        ghost_transpose(P.bc[2], g);
        r[0] += g[0]; r[2] += g[1]; r[1] += g[2]; r[3] += g[3];
      }
      if ((!pery && j == P.ny - 1) || (pery && j == 0)) {  // N ghost: right state of (i, ny - 1/2)
        const long long kk = (long long)P.ny * P.nx + i;
        for (int c = 0; c < 4; ++c) g[c] = S.fy[(4 + c) * nfy + kk];
        law_bar<GRASS>(P, S, cells, next, sve::ext_index(P, i, P.ny), true, A, m, q[2 * nall + nfx + kk],
                       q[3 * nall + nfx + kk], g, Ab, mb, Kb);
        ghost_transpose(P.bc[3], g);
        r[0] += g[0]; r[2] += g[1]; r[1] += g[2]; r[3] += g[3];
      }
    }
    lam[k] = r[0];
    lam[ncell + k] = r[1];
    lam[2 * ncell + k] = r[2];
    lam[3 * ncell + k] = r[3];
  }
  // Grass: the A_g and m_g gradients; Shields laws: the friction
  // coefficient's (through tau*)
  if (GRASS) {
    const double bA = block_sum(Ab, sh);
    const double bm = block_sum(mb, sh);
    if (threadIdx.x == 0) {
      gpart[2 * blockIdx.x] = bA;
      gpart[2 * blockIdx.x + 1] = bm;
    }
    finish_partials<kAdjThreads>(gpart, 2, gacc, done);
  } else {
    const double bK = block_sum(Kb, sh);
    if (threadIdx.x == 0) gpart[blockIdx.x] = bK;
    finish_partials<kAdjThreads>(gpart, 1, gacc + 2, done);
  }
}

#define ADJ_TRY(expr)                               \
  do {                                              \
    if ((expr) != cudaSuccess) return SVE_ERR_CUDA; \
  } while (0)

int status_of(const sve_handle* h) {
  DevScalars s;
  if (cudaMemcpyAsync(&s, h->sc, sizeof(s), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess) return SVE_ERR_CUDA;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SVE_ERR_CUDA;
  if (s.status & sve::ST_NAN) return SVE_ERR_NAN;
  if (s.status & sve::ST_NEG_DEPTH) return SVE_ERR_NEG_DEPTH;
  if (s.status & sve::ST_RIEMANN) return SVE_ERR_RIEMANN;
  if (s.status & sve::ST_DT) return SVE_ERR_DT;
  return SVE_OK;
}

// copy the 4 padded conserved fields of the handle to / from a buffer
int save_state(sve_handle* h, double* dst) {
  const size_t n = (size_t)h->next;
  for (int f = 0; f < 4; ++f)
    ADJ_TRY(cudaMemcpyAsync(dst + f * n, h->fields[f], sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream));
  return SVE_OK;
}
int load_state(sve_handle* h, const double* src) {
  const size_t n = (size_t)h->next;
  for (int f = 0; f < 4; ++f)
    ADJ_TRY(cudaMemcpyAsync(h->fields[f], src + f * n, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream));
  return SVE_OK;
}

template <typename E>
int grow(E** p, size_t* cap, size_t n) {
  if (*cap >= n) return SVE_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  if (cudaMalloc(p, sizeof(E) * n) != cudaSuccess) return SVE_ERR_OOM;
  *cap = n;
  return SVE_OK;
}

void free_rec(sve_adjoint_rec* r) {
  if (!r) return;
  for (double* c : r->checkpoints) cudaFree(c);
  if (r->kseg) cudaFree(r->kseg);
  if (r->ksegc) cudaFree(r->ksegc);
  if (r->kroots) cudaFree(r->kroots);
  if (r->krtry) cudaFree(r->krtry);
  if (r->seg) cudaFree(r->seg);
  if (r->segc) cudaFree(r->segc);
  if (r->roots) cudaFree(r->roots);
  if (r->rtry) cudaFree(r->rtry);
  if (r->cells) cudaFree(r->cells);
  if (r->q) cudaFree(r->q);
  if (r->lam) cudaFree(r->lam);
  if (r->mu) cudaFree(r->mu);
  if (r->gpart) cudaFree(r->gpart);
  if (r->gacc) cudaFree(r->gacc);
  if (r->done) cudaFree(r->done);
  delete r;
}

// One forward step with the handle's kernels: of size dt (fixed-dt mode),
// or with cfl set of the CFL size, logged in the handle's time-step log at
// the call's step counter.  With conv, the step's convected (pre-friction)
// interior state is kept there; with roots, each interface's Newton root
// and the doublings of a of its solve (roots, rtry).
int forward_step(sve_handle* h, double dt, double* conv = nullptr, bool cfl = false, double* roots = nullptr,
                 unsigned char* rtry = nullptr) {
  if (!cfl) {
    ADJ_TRY(cudaMemcpyAsync(h->fixed, &dt, sizeof(double), cudaMemcpyHostToDevice, h->stream));
    ADJ_TRY(cudaMemsetAsync(&h->sc->call_step, 0, sizeof(int), h->stream));
  }
  DevState<double> S = state_of<double>(h);
  const unsigned nbi = (unsigned)sve::iface_blocks(h->P, sve::kThreadsStep);
  const unsigned nbc = (unsigned)sve::cell_blocks(h->P, sve::kThreadsStep);
  if (roots)
    sve::interface_kernel<double, sve::kThreadsStep, true><<<nbi, sve::kThreadsStep, 0, h->stream>>>(
        h->P, S, h->sc, h->fixed, h->dtlog, cfl ? 0 : 1, roots, rtry);
  else
    sve::interface_kernel<double><<<nbi, sve::kThreadsStep, 0, h->stream>>>(h->P, S, h->sc, h->fixed, h->dtlog,
                                                                            cfl ? 0 : 1);
  if (conv) {
    const long long ncell = (long long)h->P.nx * h->P.ny;
    convect_save_kernel<<<(unsigned)((ncell + kAdjThreads - 1) / kAdjThreads), kAdjThreads, 0, h->stream>>>(
        h->P, S, h->sc, conv);
  }
  sve::cell_kernel<double><<<nbc, sve::kThreadsStep, 0, h->stream>>>(h->P, S, h->sc, h->mpart,
                                                                     sve::Mirror<double>{});
  return cudaGetLastError() == cudaSuccess ? SVE_OK : SVE_ERR_CUDA;
}

}  // namespace

__attribute__((visibility("hidden"))) void sve_internal_adjoint_free(sve_handle* h) {
  if (h && h->adj) {
    cudaStreamSynchronize(h->stream);
    free_rec(h->adj);
    h->adj = nullptr;
  }
}

__attribute__((visibility("hidden"))) bool sve_internal_has_external(const sve_config* c);

extern "C" {

int sve_record_forward(sve_handle* h, int nsteps, int checkpoint_every) {
  if (!h || nsteps < 1) return SVE_ERR_ARG;
  if (!h->has_state) return SVE_ERR_STATE;
  if (h->cfg.precision != SVE_FP64 || sve_internal_has_external(&h->cfg) || h->scheme) return SVE_ERR_ARG;
  sve_internal_adjoint_free(h);
  sve_adjoint_rec* r = new sve_adjoint_rec();
  h->adj = r;
  r->nsteps = nsteps;
  const size_t n = 4 * (size_t)h->next;
  const long long ncell = (long long)h->P.nx * h->P.ny;
  double t0 = 0.0;
  ADJ_TRY(cudaMemcpy(&t0, &h->sc->t, sizeof(double), cudaMemcpyDeviceToHost));
  r->t0 = t0;
  r->dts.resize(nsteps);
  // Automatic checkpointing, within the memory budget (sve_set_adjoint_budget;
  // by default half of the free device memory): when every step's padded
  // state, convected state and Newton roots fit, the recording keeps them
  // all and the adjoint recomputes nothing; otherwise checkpoints every
  // ceil(sqrt(N)) steps, each segment recomputed once before its reverse
  // sweep, except the last segments whose data the rest of the budget holds.
  const double nfd = (double)(h->P.nfx + h->P.nfy);
  const double per_step = (double)sizeof(double) * ((double)n + 4.0 * (double)ncell + nfd) + nfd;
  double budget = 0.0;
  if (checkpoint_every <= 0) {
    size_t free_b = 0, total_b = 0;
    ADJ_TRY(cudaMemGetInfo(&free_b, &total_b));
    budget = h->adj_budget >= 0 ? (double)h->adj_budget : 0.5 * (double)free_b;
    r->stored = per_step * (double)nsteps <= budget;
  }
  if (r->stored) {
    r->every = nsteps;
    r->ncp = 1;
    double* c = nullptr;
    int rc = cudaMalloc(&c, sizeof(double) * n) == cudaSuccess ? SVE_OK : SVE_ERR_OOM;
    if (!rc) r->checkpoints.push_back(c);
    if (!rc) rc = save_state(h, c);
    if (!rc) rc = grow(&r->seg, &r->seg_cap, n * (size_t)nsteps);
    if (!rc) rc = grow(&r->segc, &r->segc_cap, 4 * (size_t)ncell * (size_t)nsteps);
    const size_t nf = (size_t)(h->P.nfx + h->P.nfy);
    if (!rc) rc = grow(&r->roots, &r->roots_cap, nf * (size_t)nsteps);
    if (!rc) rc = grow(&r->rtry, &r->rtry_cap, nf * (size_t)nsteps);
    if (!rc) rc = sve_internal_reserve_dtlog(h, nsteps);
    if (!rc && cudaMemsetAsync(&h->sc->call_step, 0, sizeof(int), h->stream) != cudaSuccess) rc = SVE_ERR_CUDA;
    for (int s = 0; s < nsteps && !rc; ++s) {
      rc = save_state(h, r->seg + (size_t)s * n);
      if (!rc)
        rc = forward_step(h, 0.0, r->segc + (size_t)s * 4 * (size_t)ncell, true, r->roots + (size_t)s * nf,
                          r->rtry + (size_t)s * nf);
    }
    if (!rc) rc = status_of(h);
    if (!rc && cudaMemcpy(r->dts.data(), h->dtlog, sizeof(double) * (size_t)nsteps, cudaMemcpyDeviceToHost) !=
                   cudaSuccess)
      rc = SVE_ERR_CUDA;
    if (rc) { sve_internal_adjoint_free(h); return rc; }
    h->last_steps = nsteps;
    return SVE_OK;
  }
  r->every = checkpoint_every > 0 ? checkpoint_every : (int)ceil(sqrt((double)nsteps));
  if (r->every > nsteps) r->every = nsteps;
  const int ncp = (nsteps + r->every - 1) / r->every;
  r->ncp = ncp;
  r->kept_from = ncp;
  auto seg_len = [&](int k) { return (k + 1) * r->every <= nsteps ? r->every : nsteps - k * r->every; };
  if (checkpoint_every <= 0) {
    // what the budget holds beyond the checkpoints and one recomputed
    // segment of the reverse sweep, from the last segment backwards
    double rest = budget - per_step * (double)r->every - (double)sizeof(double) * (double)n * (double)ncp;
    int kept = 0;
    for (int k = ncp - 1; k >= 1; --k) {
      if (per_step * (double)(kept + seg_len(k)) > rest) break;
      kept += seg_len(k);
      r->kept_from = k;
    }
    if (kept > 0) {
      const size_t nf = (size_t)(h->P.nfx + h->P.nfy);
      size_t c0 = 0, c1 = 0, c2 = 0, c3 = 0;
      int rc = grow(&r->kseg, &c0, n * (size_t)kept);
      if (!rc) rc = grow(&r->ksegc, &c1, 4 * (size_t)ncell * (size_t)kept);
      if (!rc) rc = grow(&r->kroots, &c2, nf * (size_t)kept);
      if (!rc) rc = grow(&r->krtry, &c3, nf * (size_t)kept);
      if (rc) {  // not there after all: checkpoints only
        cudaGetLastError();
        cudaFree(r->kseg); cudaFree(r->ksegc); cudaFree(r->kroots); cudaFree(r->krtry);
        r->kseg = r->ksegc = r->kroots = nullptr;
        r->krtry = nullptr;
        r->kept_from = ncp;
      }
    }
  }
  const size_t nf = (size_t)(h->P.nfx + h->P.nfy);
  const int n0k = r->kept_from * r->every;
  for (int k = 0; k < ncp; ++k) {
    const int len = seg_len(k);
    if (k < r->kept_from) {
      double* c = nullptr;
      if (cudaMalloc(&c, sizeof(double) * n) != cudaSuccess) { sve_internal_adjoint_free(h); return SVE_ERR_OOM; }
      r->checkpoints.push_back(c);
      int rc = save_state(h, c);
      rc = rc ? rc : sve_step(h, len, nullptr);
      if (rc) { sve_internal_adjoint_free(h); return rc; }
      if (sve_get_dts(h, r->dts.data() + (size_t)k * r->every, len) != len) { sve_internal_adjoint_free(h); return SVE_ERR_CUDA; }
      continue;
    }
    // a kept segment: as the stored recording, step by step
    int rc = SVE_OK;
    if (k == r->kept_from) {
      rc = sve_internal_reserve_dtlog(h, nsteps - n0k);
      if (!rc && cudaMemsetAsync(&h->sc->call_step, 0, sizeof(int), h->stream) != cudaSuccess) rc = SVE_ERR_CUDA;
    }
    for (int s = 0; s < len && !rc; ++s) {
      const size_t g = (size_t)(k * r->every + s - n0k);
      rc = save_state(h, r->kseg + g * n);
      if (!rc) rc = forward_step(h, 0.0, r->ksegc + g * 4 * (size_t)ncell, true, r->kroots + g * nf, r->krtry + g * nf);
    }
    if (rc) { sve_internal_adjoint_free(h); return rc; }
  }
  if (r->kept_from < ncp) {
    int rc = status_of(h);
    if (!rc && cudaMemcpy(r->dts.data() + n0k, h->dtlog, sizeof(double) * (size_t)(nsteps - n0k),
                          cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = SVE_ERR_CUDA;
    if (rc) { sve_internal_adjoint_free(h); return rc; }
    h->last_steps = nsteps - n0k;
  }
  return SVE_OK;
}

int sve_get_checkpoint_every(sve_handle* h) {
  if (!h) return SVE_ERR_ARG;
  if (!h->adj) return SVE_ERR_STATE;
  return h->adj->every;
}

int sve_set_adjoint_budget(sve_handle* h, long long bytes) {
  if (!h || bytes < -1) return SVE_ERR_ARG;
  h->adj_budget = bytes;
  return SVE_OK;
}

int sve_get_adjoint_kept_steps(sve_handle* h) {
  if (!h) return SVE_ERR_ARG;
  if (!h->adj) return SVE_ERR_STATE;
  const sve_adjoint_rec* r = h->adj;
  if (r->stored) return r->nsteps;
  return r->kept_from >= r->ncp ? 0 : r->nsteps - r->kept_from * r->every;
}

int sve_adjoint(sve_handle* h, const void* lam_h, const void* lam_hu, const void* lam_hv, const void* lam_z,
                int where, void* g_h0, void* g_hu0, void* g_hv0, void* g_z0, double* g_params) {
  if (!h || (where != SVE_HOST && where != SVE_DEVICE)) return SVE_ERR_ARG;
  sve_adjoint_rec* r = h->adj;
  if (!r) return SVE_ERR_STATE;
  const DevParams& P = h->P;
  const long long ncell = (long long)P.nx * P.ny;
  const size_t nst = 4 * (size_t)h->next;
  int rc = SVE_OK;
  if (!r->lam && cudaMalloc(&r->lam, sizeof(double) * 8 * ncell) != cudaSuccess) return SVE_ERR_OOM;
  if (!r->mu && cudaMalloc(&r->mu, sizeof(double) * 4 * ncell) != cudaSuccess) return SVE_ERR_OOM;
  if (!r->gacc && cudaMalloc(&r->gacc, sizeof(double) * 4) != cudaSuccess) return SVE_ERR_OOM;
  if (!r->done && cudaMalloc(&r->done, sizeof(unsigned int)) != cudaSuccess) return SVE_ERR_OOM;
  const int nb_if = (int)((P.nfx + P.nfy + kAdjThreads - 1) / kAdjThreads);
  const int nb_c = (int)((ncell + kAdjThreads - 1) / kAdjThreads);
  rc = grow(&r->gpart, &r->gpart_cap, 2 * (size_t)(nb_if > nb_c ? nb_if : nb_c));
  if (rc) return rc;
  rc = grow(&r->seg, &r->seg_cap, nst * (size_t)r->every);
  if (rc) return rc;
  rc = grow(&r->segc, &r->segc_cap, 4 * (size_t)ncell * (size_t)r->every);
  if (rc) return rc;
  const size_t nf = (size_t)(P.nfx + P.nfy);
  rc = grow(&r->roots, &r->roots_cap, nf * (size_t)r->every);
  if (rc) return rc;
  rc = grow(&r->rtry, &r->rtry_cap, nf * (size_t)r->every);
  if (rc) return rc;
  rc = grow(&r->cells, &r->cells_cap, (size_t)kCPlanes * (size_t)h->next);
  if (rc) return rc;
  rc = grow(&r->q, &r->q_cap, 4 * nf);
  if (rc) return rc;
  const unsigned nb_pad = (unsigned)((h->next + kAdjThreads - 1) / kAdjThreads);
  double* lam = r->lam;             // lambda^{n+1}
  double* lam_next = r->lam + 4 * ncell;
  ADJ_TRY(cudaMemsetAsync(r->gacc, 0, sizeof(double) * 4, h->stream));
  ADJ_TRY(cudaMemsetAsync(r->done, 0, sizeof(unsigned int), h->stream));
  const cudaMemcpyKind kin = where == SVE_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const void* lin[4] = {lam_h, lam_hu, lam_hv, lam_z};
  for (int f = 0; f < 4; ++f) {
    if (lin[f] && !(f == 2 && P.dim == 1))
      ADJ_TRY(cudaMemcpyAsync(lam + f * ncell, lin[f], sizeof(double) * ncell, kin, h->stream));
    else
      ADJ_TRY(cudaMemsetAsync(lam + f * ncell, 0, sizeof(double) * ncell, h->stream));
  }
  DevState<double> S = state_of<double>(h);
  const unsigned nbc = (unsigned)sve::cell_blocks(P, sve::kThreads);
  const int ncp = r->ncp;
  for (int k = ncp - 1; k >= 0; --k) {
    const int n0 = k * r->every;
    const int len = (k + 1) * r->every <= r->nsteps ? r->every : r->nsteps - n0;
    // the segment's states U^{n0} .. U^{n0 + len - 1}: kept by the recording
    // (every step, or this segment), else recomputed from its checkpoint
    const double* seg = r->seg;
    const double* segc = r->segc;
    const double* kr = r->roots;
    const unsigned char* kt = r->rtry;
    if (!r->stored && k >= r->kept_from) {
      const size_t g0 = (size_t)(n0 - r->kept_from * r->every);
      seg = r->kseg + g0 * nst;
      segc = r->ksegc + g0 * 4 * (size_t)ncell;
      kr = r->kroots + g0 * nf;
      kt = r->krtry + g0 * nf;
    }
    if (!r->stored && k < r->kept_from) {
      rc = load_state(h, r->checkpoints[k]);
      if (rc) return rc;
      sve::init_kernel<double><<<nbc, sve::kThreads, 0, h->stream>>>(P, S, h->sc, h->mpart);
      for (int s = 0; s < len; ++s) {
        rc = save_state(h, r->seg + (size_t)s * nst);
        if (!rc)
          rc = forward_step(h, r->dts[n0 + s], r->segc + (size_t)s * 4 * (size_t)ncell, false,
                            r->roots + (size_t)s * nf, r->rtry + (size_t)s * nf);
        if (rc) return rc;
      }
    }
    // reverse through the segment: the saved padded state U^n (its ghosts
    // included) and its convected state are all the adjoint kernels read
    for (int s = len - 1; s >= 0; --s) {
      const double dt = r->dts[n0 + s];
      rc = load_state(h, seg + (size_t)s * nst);
      if (rc) return rc;
      adj_friction_kernel<<<nb_c, kAdjThreads, 0, h->stream>>>(P, segc + (size_t)s * 4 * (size_t)ncell, lam,
                                                              r->mu, dt, r->gpart, r->gacc, r->done);
      const double* roots = kr + (size_t)s * nf;
      const unsigned char* rtry = kt + (size_t)s * nf;
      const double A = h->cfg.A_g, m = h->cfg.m_g;
      if (P.bedload == 0) {
        adj_cells_kernel<true><<<nb_pad, kAdjThreads, 0, h->stream>>>(P, S, A, m, r->cells, h->next);
        adj_interface_kernel<true><<<nb_if, kAdjThreads, 0, h->stream>>>(P, S, r->mu, dt, A, m, roots, rtry,
                                                                         r->cells, h->next, r->q);
        adj_gather_kernel<true><<<nb_c, kAdjThreads, 0, h->stream>>>(P, S, r->mu, r->q, r->cells, h->next, A, m,
                                                                     lam_next, r->gpart, r->gacc, r->done);
      } else {
        adj_cells_kernel<false><<<nb_pad, kAdjThreads, 0, h->stream>>>(P, S, A, m, r->cells, h->next);
        adj_interface_kernel<false><<<nb_if, kAdjThreads, 0, h->stream>>>(P, S, r->mu, dt, A, m, roots, rtry,
                                                                          r->cells, h->next, r->q);
        adj_gather_kernel<false><<<nb_c, kAdjThreads, 0, h->stream>>>(P, S, r->mu, r->q, r->cells, h->next, A,
                                                                      m, lam_next, r->gpart, r->gacc, r->done);
      }
      if (cudaGetLastError() != cudaSuccess) return SVE_ERR_CUDA;
      double* t = lam;
      lam = lam_next;
      lam_next = t;
    }
  }
  // the handle holds U^0 again (the last state loaded): project it, so that
  // stepping on from here starts from a consistent state
  sve::init_kernel<double><<<nbc, sve::kThreads, 0, h->stream>>>(P, S, h->sc, h->mpart);
  rc = status_of(h);
  if (rc) return rc;
  const cudaMemcpyKind kout = where == SVE_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  void* outs[4] = {g_h0, g_hu0, g_hv0, g_z0};
  for (int f = 0; f < 4; ++f)
    if (outs[f] && !(f == 2 && P.dim == 1))
      ADJ_TRY(cudaMemcpyAsync(outs[f], lam + f * ncell, sizeof(double) * ncell, kout, h->stream));
  double g[4] = {0, 0, 0, 0};
  ADJ_TRY(cudaMemcpyAsync(g, r->gacc, sizeof(double) * 4, cudaMemcpyDeviceToHost, h->stream));
  // the handle now holds the recorded run's initial state at its time
  ADJ_TRY(cudaMemcpyAsync(&h->sc->t, &r->t0, sizeof(double), cudaMemcpyHostToDevice, h->stream));
  ADJ_TRY(cudaStreamSynchronize(h->stream));
  if (g_params) { g_params[0] = g[0]; g_params[1] = g[1]; g_params[2] = g[2]; }
  return SVE_OK;
}

}  // extern "C"
