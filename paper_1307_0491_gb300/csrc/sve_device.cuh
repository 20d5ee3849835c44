// sve_device.cuh -- device code of libsve: equilibrium projection, closures,
// the relaxation Riemann solver and the two step kernels.
//
// Step n (Sec. 3 of arXiv:1307.0491, the procedure after the list of
// properties of the relaxation model), split in two launches so that every
// floating-point operation of the method is done exactly once per step
// (GB300's FP64 pipe is ~1/58 of its FP32 pipe, so recomputation, not memory
// traffic, is what costs):
//   interface_kernel: one thread per interface (x then y) reads the projected
//     states of its two cells, solves the homogeneous relaxation Riemann
//     problem (Eqs. relaxh--relaxqs, lambda -> 0 projection already done),
//     stores the fluctuations A-dU, A+dU and reduces the extreme wave speed;
//     the last block to finish turns the speeds into the CFL time step.
//   cell_kernel: one thread per cell averages the Riemann fans (Godunov, in
//     fluctuation form), applies semi-implicit friction, checks the state,
//     projects the new state to equilibrium (Pi = g h^2 / 2, Omega = q_b)
//     for the next step, fills the ghost ring and reduces the mass sums.
// The state and its projection live in ghost-padded arrays of
// (ny + 2) x (nx + 2) cells and are updated in place.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace sve {

enum : int { ST_RIEMANN = 1, ST_NEG_DEPTH = 2, ST_NAN = 4, ST_DT = 8 };
enum : int { GHOST_PERIODIC = 0, GHOST_FREE = 1, GHOST_INFLOW_Q = 2, GHOST_INFLOW_QH = 3, GHOST_WALL = 4,
             GHOST_EXTERNAL = 5 };  // external: the ghost ring is set from outside (a neighbouring block)
// How the solve pass ends a step: the CFL step of its speeds, a given step,
// or only the block's extreme speeds (a block of a decomposed grid: the step
// comes from the maximum over all blocks).
enum : int { DT_CFL = 0, DT_FIXED = 1, DT_SPEEDS_ONLY = 2 };

// Physical and numerical constants, precomputed on the host.
struct DevParams {
  int dim, nx, ny, ex;  // ex = nx + 2 (padded row length)
  double dx, dy, inv_dx, inv_dy, g, cfl, inv_2g;
  int bedload;          // 0 Grass; 1 MPM, 2 FLvB, 3 Nielsen, 4 Ribberink, 5 Camenen
  double A_g, m_g;
  int m_int;            // m_g if it is 1, 2, 3 or 4, else 0 (pow path)
  double qs_scale;      // sqrt((s-1) g d_s^3): q_b = qs_scale q*(tau*) (Shields laws)
  double mpm_alpha;     // tau* = alpha |U|^2; Darcy: f / (8 g (s-1) d_s);  Manning: n^2 / ((s-1) d_s) (over h^(1/3))
  double tau_cr;
  int friction;         // 0 none, 1 Darcy, 2 Strickler
  double fric_c;        // Darcy: f / 8;  Strickler: g / K^2
  double fric_coef;     // the friction law's coefficient: f (Darcy) or K (Strickler)
  int bc[4];
  double q_in, h_in;
  double kappa_a, beta_min, gamma_z, newton_tol;
  double two_g, two_g_gamma;  // 2 g and 2 g gamma_z (products the solver uses)
  int newton_maxit;
  long long nfx, nfy;   // number of x- and y-interfaces
  // FP32 copies (rounded on the host) for the FP32-state kernels: converting
  // a double inside a kernel is an FP64-pipe instruction, and GB300's FP64
  // pipe is ~1/64 of its FP32 pipe
  struct {
    float g, inv_2g, A_g, m_g, qs_scale, mpm_alpha, tau_cr, fric_c, q_in, h_in, kappa_a, beta_min, gamma_z, newton_tol;
    float two_g, two_g_gamma;
  } f;
};

// Parameter x of DevParams in precision T: the double itself, or its FP32
// copy P.f.x for float (same value as (float)x).
template <typename T> __device__ __forceinline__ T par(double d, float) { return T(d); }
template <> __device__ __forceinline__ float par<float>(double, float f) { return f; }

// Device scalars of one handle.
struct DevScalars {
  double dt, t;
  double mass_h, mass_z;
  double Sx, Sy;
  int status;
  int call_step;        // step index inside the current step call
  unsigned int done_iface, done_cell;
  long long steps;      // total steps since the state was set
  unsigned long long newton_iters;  // Newton updates summed over all solves since the state was set
  unsigned long long smax_bits[2];  // running max of the x / y wave speeds of the step (bit patterns; 0 between steps)
  unsigned int mass_parts;  // per-block (h, z) partials of the last step or upload, summed on read-out (mass_kernel)
  // safeguards taken since the state was set, summed over all solves:
  // Newton steps halved to keep every tau_k positive, solves whose celerity
  // a was raised by the bed-jump bound (gamma_z), and doublings of a where
  // the bounds admitted no solution with positive tau_k
  unsigned long long halvings, raised, retries;
  unsigned long long hist_count;  // records written to the per-step history ring (sve_set_history)
};

// Ghost-padded state and projection (SoA) of precision T.
template <typename T>
struct DevState {
  T *h, *hu, *hv, *z;                        // conserved
  T *tau, *u, *v, *pi, *omx, *omy, *ca, *cbx, *cby;  // projection
  T *fx, *fy;                                // fluctuations: 8 planes (A- H,qn,qt,Z, A+ H,qn,qt,Z)
};

// Optional second destination of a step's new interior state: row-major
// ny x nx arrays (h is null when unused; hv unused in 1D).  A caller's
// page-locked host buffers go here, so that the last step of a host-to-host
// call stores its result over the host link from the cell update itself.
template <typename T>
struct Mirror {
  T *h, *hu, *hv, *z;
};

template <typename T> __device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }
template <typename T> __device__ __forceinline__ T tabs(T a) { return a < T(0) ? -a : a; }
// Quotients and square roots: IEEE in FP64; in the FP32-state path the
// hardware approximations (div.approx, sqrt.approx: ~2 ulp), whose error is
// far below what FP32 state storage already costs (the FP32 path is checked
// against the FP64 oracle with stated bounds).
__device__ __forceinline__ double tsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float tsqrt(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ double tdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float tdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double tcbrt(double x) { return cbrt(x); }
__device__ __forceinline__ float tcbrt(float x) { return cbrtf(x); }
__device__ __forceinline__ double tpow(double x, double y) { return pow(x, y); }
__device__ __forceinline__ double texp(double x) { return exp(x); }
__device__ __forceinline__ float texp(float x) { return expf(x); }
__device__ __forceinline__ float tpow(float x, float y) { return powf(x, y); }
__device__ __forceinline__ bool tfinite(double x) { return isfinite(x); }
// a b + c with one rounding, written out where a sum has two products: the
// compiler's own contraction may fuse either product, and not alike in
// every kernel that inlines the expression -- the projection of a cell runs
// in several kernels (upload, update, ghosts) that must agree bit for bit.
__device__ __forceinline__ double tfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float tfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ bool tfinite(float x) { return isfinite(x); }
// Whether a quotient is cheap enough to take several where one would do (FP32:
// div.approx); in FP64 (and its dual numbers) divides are folded into one.
template <typename T> struct cheap_div { static constexpr bool value = false; };
template <> struct cheap_div<float> { static constexpr bool value = true; };

// ---- FP64 arithmetic on GB300 -------------------------------------------
// GB300 issues about two FP64 instructions per SM clock.  Measured costs in
// DFMA issue slots: IEEE divide ~4.6, square root ~7.5, cube root ~12;
// FP64 compare, select and min/max one slot each.  Divides and square roots
// stay IEEE (Newton-Raphson refinement of FP32 seeds measured slower); the
// inverse cube root of the Strickler law is refined from an FP32 seed (it
// replaces a cube root and a divide); comparisons, |.| and max of
// non-negative values use integer operations on the bit patterns.

// x^(-1/3) for x > 0: rcbrtf seed, two Newton-Raphson steps of
// y <- y + (y/3)(1 - x y^3) (the classical iteration for the inverse cube
// root; the error e becomes ~2e^2 per step), IEEE fallback outside the FP32
// exponent range.  tests/test_gpu_arith.py compares it with 1/cbrt.
__device__ __forceinline__ bool f32_safe(double x) {
  const int e = (int)((__double_as_longlong(x) >> 52) & 0x7ff);
  return e > 1023 - 120 && e < 1023 + 120;
}
__device__ __forceinline__ double rcbrt64(double x) {
  if (!f32_safe(x)) return 1.0 / cbrt(x);
  double y = (double)rcbrtf((float)x);
  const double third = 1.0 / 3.0;
  double y3 = y * y * y;
  y = fma(third * y, fma(-x, y3, 1.0), y);
  y3 = y * y * y;
  return fma(third * y, fma(-x, y3, 1.0), y);
}
__device__ __forceinline__ float rcbrt64(float x) { return rcbrtf(x); }

// max / |.| of non-negative doubles by integer compares of the bit patterns
// (IEEE order of non-negative values is their integer order), keeping them
// off the FP64 pipe.  Not for negative or NaN arguments.
__device__ __forceinline__ double nnmax(double a, double b) {
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  return __longlong_as_double(ia > ib ? ia : ib);
}
__device__ __forceinline__ float nnmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double absbits(double a) {
  return __longlong_as_double(__double_as_longlong(a) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ float absbits(float a) { return fabsf(a); }
__device__ __forceinline__ bool positive(double a) { return __double_as_longlong(a) > 0LL; }
__device__ __forceinline__ bool positive(float a) { return a > 0.0f; }
__device__ __forceinline__ bool negative(double a) {  // a < 0 (-0.0 counts as 0)
  return __double_as_longlong(a) < 0LL && __double_as_longlong(a) != (long long)0x8000000000000000ULL;
}
__device__ __forceinline__ bool negative(float a) { return a < 0.0f; }
__device__ __forceinline__ bool finite_bits(double a) {
  return (__double_as_longlong(a) & 0x7ff0000000000000LL) != 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool finite_bits(float a) { return isfinite(a); }
__device__ __forceinline__ bool same_bits(double a, double b) {
  return __double_as_longlong(a) == __double_as_longlong(b);
}
__device__ __forceinline__ bool same_bits(float a, float b) { return __float_as_int(a) == __float_as_int(b); }

// ---- closures (Sec. 2) -----------------------------------------------------
// Non-dimensional rate q*(tau*) of the Shields-parameter laws listed in
// Sec. 2 and dq*/dtau*, x = tau* - tau*_cr; false where the law carries
// nothing (below the threshold; tau* = 0 for Camenen's).
//   1 MPM (Eq. MPM)             8 x^1.5
//   2 FLvB (Eq. FLVB)           5.7 x^1.5
//   3 Nielsen (Eq. Nielsen)     12 sqrt(tau*) x
//   4 Ribberink (Eq. Ribberink) 11 x^1.65
//   5 Camenen (Eq. Camenen)     12 tau*^1.5 exp(-4.5 tau*_cr / tau*)
template <typename T>
__device__ __forceinline__ bool shields_rate(const DevParams& P, T ts, T& q, T& dq) {
  const T tcr = par<T>(P.tau_cr, P.f.tau_cr);
  if (P.bedload == 5) {
    if (!(ts > T(0))) return false;
    const T r = tdiv(tcr, ts);
    const T sts = tsqrt(ts);
    const T e = texp(T(-4.5) * r);
    q = T(12) * ts * sts * e;
    dq = T(12) * e * tfma(T(1.5), sts, T(4.5) * tcr * tdiv(T(1), sts));
    return true;
  }
  const T x = ts - tcr;
  if (!(x > T(0))) return false;
  switch (P.bedload) {
    case 1: { const T sx = tsqrt(x); q = T(8) * x * sx; dq = T(8) * T(1.5) * sx; return true; }
    case 2: { const T sx = tsqrt(x); q = T(5.7) * x * sx; dq = T(5.7) * T(1.5) * sx; return true; }
    case 3: {
      const T sts = tsqrt(ts);
      q = T(12) * sts * x;
      dq = T(12) * (tdiv(x, T(2) * sts) + sts);
      return true;
    }
    case 4: { q = T(11) * tpow(x, T(1.65)); dq = T(1.65) * tdiv(q, x); return true; }
    default: return false;
  }
}
// Normal bedload flux Q = q_b . n and dQ/du_n at fixed h.
// Grass (Eq. bedload Grass, 2D form): Q = A_g un |U|^(m-1),
//   dQ/dun = A_g (|U|^(m-1) + (m-1) un^2 |U|^(m-3)).
// Shields-parameter laws: Q = sqrt((s-1) g d_s^3) q*(tau*) un/|U|,
// tau* = alpha |U|^2 (q* above).
template <typename T>
__device__ __forceinline__ void closure(const DevParams& P, T H, T un, T ut, T& Q, T& dQ) {
  const T speed2 = tfma(un, un, ut * ut);
  if (P.bedload == 0) {
    const T A = par<T>(P.A_g, P.f.A_g);
    if (speed2 == T(0)) {
      Q = T(0);
      dQ = (P.m_int == 1) ? A : T(0);
      return;
    }
    // |U|^(m-1) and the second term (m-1) un^2 |U|^(m-3) of dQ/dun
    T pm1, d;
    switch (P.m_int) {
      case 1: pm1 = T(1); d = T(1); break;
      case 2: { T sp = tsqrt(speed2); pm1 = sp; d = pm1 + tdiv(un * un, sp); } break;
      case 3: pm1 = speed2; d = tfma(T(2), un * un, pm1); break;
      case 4: { T sp = tsqrt(speed2); pm1 = speed2 * sp; d = tfma(T(3) * (un * un), sp, pm1); } break;
      default: {
        T sp = tsqrt(speed2);
        T m = par<T>(P.m_g, P.f.m_g);
        pm1 = tpow(sp, m - T(1));
        d = tfma((m - T(1)) * (un * un), tpow(sp, m - T(3)), pm1);
      }
    }
    Q = A * un * pm1;
    dQ = A * d;
    return;
  }
  T alpha = par<T>(P.mpm_alpha, P.f.mpm_alpha);
  if (P.friction != 1) alpha = alpha * rcbrt64(H);
  T q, dq;
  if (speed2 == T(0) || !shields_rate(P, alpha * speed2, q, dq)) {
    Q = T(0);
    dQ = T(0);
    return;
  }
  const T sp = tsqrt(speed2);
  const T isp = tdiv(T(1), sp);
  const T C = par<T>(P.qs_scale, P.f.qs_scale);
  Q = C * q * (un * isp);
  // d/dun [q*(alpha |U|^2) un/|U|] = q*' 2 alpha un^2/|U| + q* ut^2/|U|^3
  dQ = C * tfma(T(2) * dq * alpha * (un * un), isp, q * (ut * ut) * (isp * isp * isp));
}

// Both normal directions of a 2D cell at once: (Qx, dQx/du) along x and
// (Qy, dQy/dv) along y share |U|, the Grass power or tau*, q*(tau*) and
// 1/|U|; only the final products differ.  Same values as two closure()
// calls up to rounding order.
template <typename T>
__device__ __forceinline__ void closure2(const DevParams& P, T H, T u, T v, T& Qx, T& dQx, T& Qy, T& dQy) {
  const T speed2 = tfma(u, u, v * v);
  if (P.bedload == 0) {
    const T A = par<T>(P.A_g, P.f.A_g);
    if (speed2 == T(0)) {
      Qx = T(0);
      Qy = T(0);
      dQx = dQy = (P.m_int == 1) ? A : T(0);
      return;
    }
    T pm1, f;  // |U|^(m-1) and (m-1) |U|^(m-3)
    switch (P.m_int) {
      case 1: pm1 = T(1); f = T(0); break;
      case 2: { T sp = tsqrt(speed2); pm1 = sp; f = tdiv(T(1), sp); } break;
      case 3: pm1 = speed2; f = T(2); break;
      case 4: { T sp = tsqrt(speed2); pm1 = speed2 * sp; f = T(3) * sp; } break;
      default: {
        T sp = tsqrt(speed2);
        T m = par<T>(P.m_g, P.f.m_g);
        pm1 = tpow(sp, m - T(1));
        f = (m - T(1)) * tpow(sp, m - T(3));
      }
    }
    Qx = A * u * pm1;
    dQx = A * tfma(u * u, f, pm1);
    Qy = A * v * pm1;
    dQy = A * tfma(v * v, f, pm1);
    return;
  }
  T alpha = par<T>(P.mpm_alpha, P.f.mpm_alpha);
  if (P.friction != 1) alpha = alpha * rcbrt64(H);
  T q, dq;
  if (speed2 == T(0) || !shields_rate(P, alpha * speed2, q, dq)) {
    Qx = Qy = dQx = dQy = T(0);
    return;
  }
  const T sp = tsqrt(speed2);
  const T isp = tdiv(T(1), sp);
  const T C = par<T>(P.qs_scale, P.f.qs_scale);
  const T isp3 = isp * isp * isp;
  const T cq = C * q, c2 = C * (T(2) * dq * alpha) * isp;
  Qx = cq * (u * isp);
  Qy = cq * (v * isp);
  dQx = tfma(c2, u * u, cq * (v * v) * isp3);
  dQy = tfma(c2, v * v, cq * (u * u) * isp3);
}

// Projected cell in the frame of one interface: n = normal, t = tangential.
template <typename T>
struct Cell {
  T H, Hn, Ht, Z;        // conserved
  T tau, un, ut, Pi, Om, ca, cb;
};

// ---- relaxation Riemann solver --------------------------------------------
// Five linearly degenerate waves u - a tau, u - b tau, u, u + b tau, u + a tau
// (tau = 1/H).  Riemann invariants (derived from Eqs. relaxh--relaxqs):
//   a-waves: u -+ a tau, Pi + a^2 tau, Z, Omega
//   b-waves: u -+ b tau, Pi + a^2 tau, Z - K tau^2, Omega - lambda Z,
//            K = (a^2 - b^2)/(2g)
//   contact: u, Pi, Z, Omega.
// Writing W1..W4 through them leaves p = tau1 + tau4, fixed by continuity of
// Omega across the contact, F(p) = 0, solved by a safeguarded Newton
// iteration started from the root of the fluid part alone (the Suliciu
// solution).  Returns false if no solution with positive tau_k was found.
// Per-interface constants of the Newton iteration.
template <typename T>
struct NewtonConst {
  T a, b, K, inv_a, inv_b, inv_K, D, C0, dZ, dsig, dN;
  // combinations the evaluation uses as they are (loop invariants of the
  // Newton iteration): sigma = s0 + dsig p, tau2,3 = sigma/2 -+ hD,
  // m = -(N / K) / p with N / K = dZK + D sigma (N = dZ + KD sigma),
  // lam2 = lam1 + amb tau1, lam4 = lam5 - amb tau4 (amb = a - b),
  // F = (lam2 - lam4) zl + (dOm + lam4 dZ); F' uses dNK = dN / K = D dsig;
  // the fan uses a2 = a^2
  T s0, hD, KD, lam1, lam5, dOm, amb;
  T dZK, dNK, a2;
};

// The intermediate states as functions of p (every invariant relation of the
// a- and b-waves and the contact holds for any p) and the residual F(p) of
// the one remaining condition, continuity of Omega across the contact.
// (u1, u4, Zs, zr: set by newton_fill, for the states at the root only.)
template <typename T>
struct NewtonEval {
  T tau1, tau2, tau3, tau4, u1, u4, lam2, lam4, Zs, F;
  T m, ip, zl, zr, dl;  // kept for F'(p); dl = lam2 - lam4
};

// The states at p given m = tau1 - tau4 and 1/p (e.tau2, e.tau3 set): what
// F needs -- the b-wave speeds lam2 = u1 - b tau1 = lam1 + (a - b) tau1 and
// lam4 = lam5 - (a - b) tau4, the bed jump zl = Z* - ZL = K (tau2^2 -
// tau1^2); with zr = Z* - ZR = zl - (ZR - ZL), F = dOm + lam2 zl - lam4 zr =
// (lam2 - lam4) zl + (dOm + lam4 dZ).
template <typename T>
__device__ __forceinline__ void newton_states(T p, const NewtonConst<T>& c, const Cell<T>& L, const Cell<T>& R,
                                              NewtonEval<T>& e) {
  const T hp = T(0.5) * p;
  e.tau1 = hp + T(0.5) * e.m;
  e.tau4 = hp - T(0.5) * e.m;
  e.lam2 = c.lam1 + c.amb * e.tau1;
  e.lam4 = c.lam5 - c.amb * e.tau4;
  e.zl = c.K * (e.tau2 * e.tau2 - e.tau1 * e.tau1);
  e.dl = e.lam2 - e.lam4;
  e.F = e.dl * e.zl + (c.dOm + e.lam4 * c.dZ);
}

// The rest of the states at an evaluated point: the velocities u1 = uL + a
// (tau1 - tauL) = lam1 + a tau1 and u4 = lam5 - a tau4, Z* = ZL + zl and
// zr = Z* - ZR = zl - dZ.
template <typename T>
__device__ __forceinline__ void newton_fill(const NewtonConst<T>& c, const Cell<T>& L, NewtonEval<T>& e) {
  e.u1 = c.lam1 + c.a * e.tau1;
  e.u4 = c.lam5 - c.a * e.tau4;
  e.Zs = L.Z + e.zl;
  e.zr = e.zl - c.dZ;
}

template <typename T>
__device__ __forceinline__ void newton_sigma(T p, const NewtonConst<T>& c, NewtonEval<T>& e, T& sigma) {
  sigma = c.s0 + c.dsig * p;                        // from u* continuity: (C0 - (a - b) p) / b
  e.tau2 = T(0.5) * sigma - c.hD;                   // from Pi continuity: (sigma -+ D) / 2
  e.tau3 = T(0.5) * sigma + c.hD;
}

// The states and F at p, with ip = 1/p given.
template <typename T>
__device__ __forceinline__ void newton_eval_ip(T p, T ip, const NewtonConst<T>& c, const Cell<T>& L,
                                               const Cell<T>& R, NewtonEval<T>& e) {
  T sigma;
  newton_sigma(p, c, e, sigma);
  e.ip = ip;
  e.m = -(c.dZK + c.D * sigma) * ip;                // from Z* continuity: -N / (K p)
  newton_states(p, c, L, R, e);
}

template <typename T>
__device__ __forceinline__ void newton_eval(T p, const NewtonConst<T>& c, const Cell<T>& L, const Cell<T>& R,
                                            NewtonEval<T>& e) {
  newton_eval_ip(p, tdiv(T(1), p), c, L, R, e);
}

// Analytic F'(p) at an evaluated point.
template <typename T>
__device__ __forceinline__ T newton_deriv(const NewtonConst<T>& c, const NewtonEval<T>& e, T& dm) {
  dm = -(c.dNK + e.m) * e.ip;                       // (-dN/K - m) / p
  // dtau1,4/dp = (1 +- dm)/2, dtau2,3/dp = dsig/2:
  // dZ*/dp = 2K (tau2 dsig/2 - tau1 (1 + dm)/2)
  const T dZs = c.K * (c.dsig * e.tau2 - e.tau1 * (T(1) + dm));
  // (a - b) (dtau1 zl + dtau4 zr) + (lam2 - lam4) dZs, where dtau1 zl +
  // dtau4 zr = zl + (dm - 1) dZ / 2 (zr = zl - dZ)
  return c.amb * (e.zl + (T(0.5) * dm - T(0.5)) * c.dZ) + e.dl * dZs;
}

template <typename T>
__device__ __forceinline__ T newton_deriv(const NewtonConst<T>& c, const NewtonEval<T>& e) {
  T dm;
  return newton_deriv(c, e, dm);
}

template <typename T>
__device__ __forceinline__ bool newton_positive(const NewtonEval<T>& e) {
  return positive(e.tau1) && positive(e.tau2) && positive(e.tau3) && positive(e.tau4);
}

// |x| <= y for y >= 0 on the bit patterns (integer compare, off the FP64 pipe).
__device__ __forceinline__ bool abs_le(double x, double y) {
  return (__double_as_longlong(x) & 0x7fffffffffffffffLL) <= __double_as_longlong(y);
}
__device__ __forceinline__ bool abs_le(float x, float y) { return fabsf(x) <= y; }

// Safeguarded Newton from the evaluated point (p, e): steps that would make
// a tau_k non-positive are halved (at most 60 times); stops after a full
// (unhalved) step with |step| <= tol p -- a halved step is short because the
// iterate is at the edge of the admissible set, not because it is near the
// root, so it never ends the iteration.  iters is incremented per accepted
// update, halv by the halvings of the accepted updates.
//
// The update that meets the stopping rule takes the states at p + step as
// first-order updates of those at p (m by dm/dp, 1/p by -1/p^2; tau2, tau3
// exact), an O(tol^2) difference from a full evaluation -- no divide.  In
// FP32, where instruction issue bounds the solve, the lanes of a warp on
// either side of the rule evaluate the states at p + step in one code path
// (only m and 1/p differ); in FP64, where the FP64 pipe bounds it, the
// separate paths measured faster (C2 interface kernel 0.383 ms against
// 0.391 ms), the converged lanes' path first.
template <typename T> struct shared_update { static constexpr bool value = false; };
template <> struct shared_update<float> { static constexpr bool value = true; };

template <typename T>
__device__ __forceinline__ bool newton_loop(const NewtonConst<T>& c, const Cell<T>& L, const Cell<T>& R, T& p,
                                            NewtonEval<T>& e, int maxit, T tol, int& iters, int& halv) {
  for (int it = 0; it < maxit; ++it) {
    T dm;
    T step = tdiv(-e.F, newton_deriv(c, e, dm));
    if (!finite_bits(step)) return false;
    NewtonEval<T> tr;
    const T pn = p + step;
    const bool conv = abs_le(step, tol * pn);
    int h = 0;
    if constexpr (shared_update<T>::value) {
      T sigma;
      newton_sigma(pn, c, tr, sigma);
      if (conv) {
        tr.m = e.m + dm * step;
        tr.ip = e.ip - (e.ip * e.ip) * step;
      } else {
        tr.ip = tdiv(T(1), pn);
        tr.m = -(c.dZK + c.D * sigma) * tr.ip;
      }
      newton_states(pn, c, L, R, tr);
      if (newton_positive(tr)) {
        p = pn;
        e = tr;
        ++iters;
        if (conv) return true;
        continue;
      }
      // not admissible: a step that met the rule is evaluated in full next,
      // any other one is halved
      if (!conv) {
        h = 1;
        step = T(0.5) * step;
      }
    } else {
      if (conv) {
        T sigma;
        newton_sigma(pn, c, tr, sigma);
        tr.m = e.m + dm * step;
        tr.ip = e.ip - (e.ip * e.ip) * step;
        newton_states(pn, c, L, R, tr);
        if (newton_positive(tr)) {
          p = pn;
          e = tr;
          ++iters;
          return true;
        }
      }
    }
    for (; h <= 60; ++h) {
      newton_eval(p + step, c, L, R, tr);
      if (newton_positive(tr)) break;
      step = T(0.5) * step;
    }
    if (h > 60) return false;
    p = p + step;
    e = tr;
    ++iters;
    halv += h;
    if (h == 0 && abs_le(step, tol * p)) return true;
  }
  return false;
}
template <typename T>
__device__ __forceinline__ bool newton_loop(const NewtonConst<T>& c, const Cell<T>& L, const Cell<T>& R, T& p,
                                            NewtonEval<T>& e, int maxit, T tol, int& iters) {
  int halv = 0;
  return newton_loop(c, L, R, p, e, maxit, tol, iters, halv);
}

template <typename T> __device__ __forceinline__ T eps_of();
template <> __device__ __forceinline__ double eps_of<double>() { return 2.220446049250313e-16; }
template <> __device__ __forceinline__ float eps_of<float>() { return 1.1920929e-7f; }
// Smallest usable relative Newton step: 16 eps in FP64; 64 eps (7.6e-6) in
// FP32, where the iterates' rounding noise reaches a few eps (quadratic
// convergence leaves ~25 (7.6e-6)^2 ~ 1e-9 behind, far below FP32 rounding).
template <typename T> __device__ __forceinline__ T newton_floor();
template <> __device__ __forceinline__ double newton_floor<double>() { return 16.0 * 2.220446049250313e-16; }
template <> __device__ __forceinline__ float newton_floor<float>() { return 64.0f * 1.1920929e-7f; }

// Root of F for one interface, from p0 (the root of the fluid part alone).
// Returns false if no root with positive tau_k was reached.
// ip0 = 1/p0.
template <typename T>
__device__ __forceinline__ bool newton_root(const DevParams& P, const NewtonConst<T>& c, const Cell<T>& L,
                                            const Cell<T>& R, T p0, T ip0, NewtonEval<T>& e, int& iters,
                                            int& halv, T& p) {
  const T tol = tmax(par<T>(P.newton_tol, P.f.newton_tol), newton_floor<T>());
  p = p0;
  newton_eval_ip(p, ip0, c, L, R, e);
  return newton_loop(c, L, R, p, e, P.newton_maxit, tol, iters, halv);
}

// Celerities of one interface: the bounds of Eq. (ab) over both states,
// a scaled by kappa_a, b floored at beta_min a0, and a raised so that
// K tau_min^2 >= gamma_z |dZ| (the sediment waves can carry the bed jump).
// Returns whether that last bound raised a.
template <typename T>
__device__ __forceinline__ bool celerities(const DevParams& P, const Cell<T>& L, const Cell<T>& R, T& a, T& b) {
  const T g = par<T>(P.g, P.f.g);
  const T a0 = nnmax(L.ca, R.ca);
  const T b0 = nnmax(L.cb, R.cb);
  a = par<T>(P.kappa_a, P.f.kappa_a) * nnmax(a0, b0);
  b = nnmax(b0, par<T>(P.beta_min, P.f.beta_min) * a0);
  const T Hmax = nnmax(L.H, R.H);
  const T need = b * b + par<T>(P.two_g_gamma, P.f.two_g_gamma) * (absbits(R.Z - L.Z) * (Hmax * Hmax));
  const bool raised = a * a < need;
  if (raised) a = tsqrt(need);
  return raised;
}

// Constants of the Newton iteration; returns its start p0, the root of the
// fluid part alone (Suliciu), p = sigma; *ip0 (if given) receives 1/p0.
template <typename T>
__device__ __forceinline__ T newton_setup(const DevParams& P, const Cell<T>& L, const Cell<T>& R, T a, T b,
                                          NewtonConst<T>& c, T* ip0 = nullptr) {
  const T g = par<T>(P.g, P.f.g);
  const T ab = a * b;
  c.a2 = a * a;
  const T a2mb2 = c.a2 - b * b;
  const T du = R.un - L.un;
  c.C0 = du + a * (L.tau + R.tau);  // a p0
  T rab;
  if constexpr (cheap_div<T>::value) {
    rab = tdiv(T(1), ab);
    c.inv_K = tdiv(par<T>(P.two_g, P.f.two_g), a2mb2);
  } else if (ip0) {
    // one divide for 1/a, 1/b, 1/K (a^2 - b^2 >= (1 - 1/kappa_a^2) a^2 > 0)
    // and 1/p0 = a / C0
    const T q = ab * a2mb2;
    const T r = tdiv(T(1), q * c.C0);
    const T rq = r * c.C0;
    rab = rq * a2mb2;
    c.inv_K = par<T>(P.two_g, P.f.two_g) * (ab * rq);
    *ip0 = a * (r * q);
  } else {
    // one divide for 1/a, 1/b and 1/K
    const T r = tdiv(T(1), ab * a2mb2);
    rab = r * a2mb2;
    c.inv_K = par<T>(P.two_g, P.f.two_g) * (ab * r);
  }
  const T inv_a = b * rab;
  c.a = a;
  c.b = b;
  c.inv_a = inv_a;
  c.inv_b = a * rab;
  c.K = a2mb2 * par<T>(P.inv_2g, P.f.inv_2g);
  c.D = (R.tau - L.tau) + (R.Pi - L.Pi) * (inv_a * inv_a);
  c.dZ = R.Z - L.Z;
  c.amb = a - b;
  c.dsig = -c.amb * c.inv_b;
  c.KD = c.K * c.D;
  c.dN = c.KD * c.dsig;
  c.dZK = c.dZ * c.inv_K;
  c.dNK = c.D * c.dsig;  // dN / K (K inv_K = 1)
  c.s0 = c.C0 * c.inv_b;
  c.hD = T(0.5) * c.D;
  c.lam1 = L.un - a * L.tau;
  c.lam5 = R.un + a * R.tau;
  c.dOm = L.Om - R.Om;
  const T p0 = L.tau + R.tau + du * inv_a;
  if constexpr (cheap_div<T>::value) {
    if (ip0) *ip0 = tdiv(T(1), p0);
  }
  return p0;
}

// State m of the fan (0 = L, 1..4 = W1..W4, 5 = R: the state after the
// last wave of negative speed) from the signs of lam1, lam2, u*, lam4, lam5,
// by the rule fan_fluctuations selects with.
__device__ __forceinline__ int fan_state(bool n1, bool n2, bool n3, bool n4, bool n5) {
  return !n1 ? 0 : (n5 ? 5 : (n4 ? 4 : (n3 ? 3 : (n2 ? 2 : 1))));
}

// Fluctuations A- = sum_{lam_k < 0} lam_k [U]_k and A+ = sum_{lam_k >= 0}
// lam_k [U]_k over the five waves of the fan evaluated at e, U = (H, H un,
// H ut, Z), written with the jump relations every wave of the fan satisfies
// (for any p): lam [H] = [H un], lam [H ut] = [H un ut], lam [H un] =
// [H un^2 + Pi] + g Hbar [Z] (Hbar = 2/(tau- + tau+), nonzero [Z] only at the
// b-waves), lam [Z] at the b-waves.  With m = the number of waves of negative
// speed, the minus sums telescope to (flux of state m) - (flux of L): one
// divide for H_m and one per b-wave instead of one per intermediate state.
template <typename T>
__device__ __forceinline__ void fan_fluctuations(const DevParams& P, const Cell<T>& L, const Cell<T>& R,
                                                 const NewtonConst<T>& c, const NewtonEval<T>& e, T Am[4], T Ap[4]) {
  const T g = par<T>(P.g, P.f.g);
  const T a = c.a, b = c.b;
  const T lam1 = c.lam1;
  const T lam5 = c.lam5;
  const T u1 = c.lam1 + a * e.tau1, u4 = c.lam5 - a * e.tau4;
  const T us = u1 + b * (e.tau2 - e.tau1);
  const T lam2 = e.lam2, lam4 = e.lam4;
  // The fan's speeds are ordered (lam1 < lam2 < u* < lam4 < lam5 for
  // positive tau_k and a > b), so state m follows from the signs of the
  // speeds directly: m = 0 (L) if lam1 >= 0, else 5 (R) if lam5 < 0, else
  // the highest k in 4, 3, 2 whose wave (lam4, u*, lam2) is negative, else 1
  // (fan_state; the same rule wherever rounding breaks the order).
  const bool n1 = negative(lam1), n2 = negative(lam2), n3 = negative(us), n4 = negative(lam4),
             n5 = negative(lam5);
  const T a2 = c.a2;
  // flux (H un, H un^2 + Pi, H un ut) of L, R and of the state m
  const T FhL = L.Hn, FqL = L.Hn * L.un + L.Pi, FvL = L.Hn * L.ut;
  const T FhR = R.Hn, FqR = R.Hn * R.un + R.Pi, FvR = R.Hn * R.ut;
  T Fh, Fq, Fv;
  T tkv = T(1), ukv = T(0), vkv = T(0), Pkv = T(0);  // state m (m = 1..4)
  const bool inner = n1 && !n5;
  if (!n1) {
    Fh = FhL; Fq = FqL; Fv = FvL;
  } else if (n5) {
    Fh = FhR; Fq = FqR; Fv = FvR;
  } else {
    // W1, W2 carry the left tangential velocity and Pi_L + a^2 (tau_L - tau);
    // W3, W4 the right ones
    const bool right = n3 || n4;  // m = 3 or 4
    const T tk = n4 ? e.tau4 : (n3 ? e.tau3 : (n2 ? e.tau2 : e.tau1));
    const T uk = n4 ? u4 : ((n2 || n3) ? us : u1);
    tkv = tk;
    ukv = uk;
    vkv = right ? R.ut : L.ut;
    Pkv = (right ? R.Pi : L.Pi) + a2 * ((right ? R.tau : L.tau) - tk);
  }
  // b-waves: bed jumps and the non-conservative source g Hbar [Z]; one
  // divide for 1/tau_k, 1/(tau1 + tau2) and 1/(tau3 + tau4)
  const T zj2 = e.zl, zj4 = c.dZ - e.zl;  // Z* - ZL, ZR - Z*
  const T d12 = e.tau1 + e.tau2, d34 = e.tau3 + e.tau4;
  const T g2 = par<T>(P.two_g, P.f.two_g);
  T S2, S4, Hk;
  if constexpr (cheap_div<T>::value) {
    S2 = tdiv(g2 * zj2, d12);
    S4 = tdiv(g2 * zj4, d34);
    Hk = tdiv(T(1), tkv);
  } else {
    const T d1234 = d12 * d34;
    const T r = tdiv(T(1), tkv * d1234);
    const T grt = g2 * (r * tkv);
    S2 = zj2 * (grt * d34);
    S4 = zj4 * (grt * d12);
    Hk = r * d1234;
  }
  if (inner) {
    Fh = Hk * ukv;
    Fq = Fh * ukv + Pkv;
    Fv = Fh * vkv;
  }
  Am[0] = Fh - FhL;
  Ap[0] = FhR - Fh;
  Am[1] = (Fq - FqL) + ((n2 ? S2 : T(0)) + (n4 ? S4 : T(0)));
  Ap[1] = (FqR - Fq) + ((n2 ? T(0) : S2) + (n4 ? T(0) : S4));
  Am[2] = Fv - FvL;
  Ap[2] = FvR - Fv;
  Am[3] = (n2 ? lam2 * zj2 : T(0)) + (n4 ? lam4 * zj4 : T(0));
  Ap[3] = (n2 ? T(0) : lam2 * zj2) + (n4 ? T(0) : lam4 * zj4);
}

// The safeguards one solve took, packed into an int ("branch"): bit 0 = the
// bed-jump bound raised a, bits 1-2 = doublings of a, bits 3.. = halved
// Newton steps.
__device__ __forceinline__ unsigned branch_raised(int br) { return (unsigned)(br & 1); }
__device__ __forceinline__ unsigned branch_retries(int br) { return (unsigned)((br >> 1) & 3); }
__device__ __forceinline__ unsigned branch_halvings(int br) { return (unsigned)(br >> 3); }

// Doublings of a allowed where the celerities admit no root with positive
// tau_k (the paper's remark after Eq. (ab): stronger bounds may be needed).
constexpr int kARetries = 3;

// iters receives the number of Newton updates (0 for identical states);
// branch the safeguards taken (branch_raised, _retries, _halvings); smax the
// extreme wave speed max(|lambda1|, |lambda5|) with the celerity a used;
// pstar (if given) the root p = tau1 + tau4 reached (0 for identical states).
template <typename T>
__device__ bool riemann_solve(const DevParams& P, const Cell<T>& L, const Cell<T>& R, T Am[4], T Ap[4], T& smax,
                              int& iters, int& branch, T* pstar = nullptr) {
  iters = 0;
  T a, b;
  const bool raised = celerities(P, L, R, a, b);
  branch = raised ? 1 : 0;
  smax = nnmax(absbits(L.un - a * L.tau), absbits(R.un + a * R.tau));
#pragma unroll
  for (int c = 0; c < 4; ++c) { Am[c] = T(0); Ap[c] = T(0); }
  if (pstar) *pstar = T(0);
  if (same_bits(L.H, R.H) && same_bits(L.Hn, R.Hn) && same_bits(L.Ht, R.Ht) && same_bits(L.Z, R.Z)) return true;
  NewtonConst<T> c;
  NewtonEval<T> e;
  int halv = 0, retries = 0;
  bool ok;
  T p;
  // where the celerities admit no root with positive tau_k, a is doubled and
  // the iteration restarted (at most kARetries times; one loop, so that the
  // common single pass costs no extra registers)
  for (;;) {
    T ip0;
    const T p0 = newton_setup(P, L, R, a, b, c, &ip0);
    ok = newton_root(P, c, L, R, p0, ip0, e, iters, halv, p) && newton_positive(e);
    if (ok || retries == kARetries) break;
    ++retries;
    a = T(2) * a;
  }
  if (retries) smax = nnmax(absbits(L.un - a * L.tau), absbits(R.un + a * R.tau));
  branch += 2 * retries + 8 * halv;
  if (!ok) return false;
  if (pstar) *pstar = p;
  fan_fluctuations(P, L, R, c, e, Am, Ap);
  return true;
}

// ---- ghost cells ----------------------------------------------------------
// Ghost state of side s (0 W, 1 E, 2 S, 3 N) from the adjacent (or periodic
// partner) state in = (H, Hu, Hv, Z).
template <typename T>
__device__ __forceinline__ void ghost_state(const DevParams& P, int s, const T in[4], T out[4]) {
  const int normal = (s < 2) ? 1 : 2;
  const int tangent = (s < 2) ? 2 : 1;
  const T inward = (s == 0 || s == 2) ? T(1) : T(-1);
#pragma unroll
  for (int c = 0; c < 4; ++c) out[c] = in[c];
  switch (P.bc[s]) {
    case GHOST_INFLOW_Q: out[normal] = inward * par<T>(P.q_in, P.f.q_in); out[tangent] = T(0); break;
    case GHOST_INFLOW_QH: out[0] = par<T>(P.h_in, P.f.h_in); out[normal] = inward * par<T>(P.q_in, P.f.q_in); out[tangent] = T(0); break;
    case GHOST_WALL: out[normal] = -in[normal]; break;
    default: break;
  }
}

// Project conserved (H, Hu, Hv, Z) and store state + projection at ext index e.
template <typename T>
__device__ __forceinline__ void store_cell(const DevParams& P, const DevState<T>& S, long long e, const T s[4],
                                           T tau) {
  const T H = s[0];
  const T u = s[1] * tau;
  const T v = s[2] * tau;
  T Qx, dQx, Qy = T(0), dQy = T(0);
  if (P.dim == 2) closure2(P, H, u, v, Qx, dQx, Qy, dQy);
  else closure(P, H, u, v, Qx, dQx);
  const T g = par<T>(P.g, P.f.g);
  const T gH = g * H, gHH = gH * H;
  S.h[e] = H; S.hu[e] = s[1]; S.hv[e] = s[2]; S.z[e] = s[3];
  S.tau[e] = tau; S.u[e] = u; S.v[e] = v;
  S.pi[e] = T(0.5) * gHH;
  S.omx[e] = Qx; S.omy[e] = Qy;
  S.ca[e] = H * tsqrt(gH);
  S.cbx[e] = tsqrt(tfma(s[1], s[1], gHH * dQx));
  S.cby[e] = P.dim == 2 ? tsqrt(tfma(s[2], s[2], gHH * dQy)) : T(0);
}

__device__ __forceinline__ long long ext_index(const DevParams& P, int i, int j) {
  return (long long)(j + 1) * P.ex + (i + 1);
}

// Write the ghosts that the interior cell (i, j) with new state s feeds
// (external sides are left to the caller).
template <typename T>
__device__ __forceinline__ void write_ghosts(const DevParams& P, const DevState<T>& S, int i, int j, const T s[4]) {
  T gs[4];
  const bool perx = P.bc[0] == GHOST_PERIODIC;
  if (((!perx && i == 0) || (perx && i == P.nx - 1)) && P.bc[0] != GHOST_EXTERNAL) {
    ghost_state(P, 0, s, gs);
    store_cell(P, S, ext_index(P, -1, j), gs, tdiv(T(1), gs[0]));
  }
  if (((!perx && i == P.nx - 1) || (perx && i == 0)) && P.bc[1] != GHOST_EXTERNAL) {
    ghost_state(P, 1, s, gs);
    store_cell(P, S, ext_index(P, P.nx, j), gs, tdiv(T(1), gs[0]));
  }
  if (P.dim == 2) {
    const bool pery = P.bc[2] == GHOST_PERIODIC;
    if (((!pery && j == 0) || (pery && j == P.ny - 1)) && P.bc[2] != GHOST_EXTERNAL) {
      ghost_state(P, 2, s, gs);
      store_cell(P, S, ext_index(P, i, -1), gs, tdiv(T(1), gs[0]));
    }
    if (((!pery && j == P.ny - 1) || (pery && j == 0)) && P.bc[3] != GHOST_EXTERNAL) {
      ghost_state(P, 3, s, gs);
      store_cell(P, S, ext_index(P, i, P.ny), gs, tdiv(T(1), gs[0]));
    }
  }
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int NT>
__device__ __forceinline__ double block_max(double v, double* sh) {
  v = warp_max(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
    r = sh[0];
    for (int k = 1; k < NT / 32; ++k) r = fmax(r, sh[k]);
  }
  __syncthreads();
  return r;
}

// Block sums of (a, b), valid in thread 0, in a fixed order.  The values go
// through shared memory and one warp adds them (NT/32 serial adds per lane,
// then a shuffle tree): a shuffle tree in every warp would cost each thread
// five FP64 adds per value on GB300's narrow FP64 pipe.
template <int NT>
__device__ __forceinline__ void block_sum2(double& a, double& b, double* sh) {
  static_assert(NT % 32 == 0, "whole warps");
  __shared__ double buf[2][NT];
  buf[0][threadIdx.x] = a;
  buf[1][threadIdx.x] = b;
  __syncthreads();
  if (threadIdx.x < 32) {
    double ra = 0.0, rb = 0.0;
#pragma unroll
    for (int k = 0; k < NT / 32; ++k) { ra += buf[0][threadIdx.x + 32 * k]; rb += buf[1][threadIdx.x + 32 * k]; }
    a = warp_sum(ra);
    b = warp_sum(rb);
  }
  __syncthreads();
  (void)sh;
}

// Sum of the per-block (h, z) partials by the last block: thread t adds
// blocks t, t + NT, ... in order, then a fixed shuffle tree -- the same
// order on every run (deterministic), with no serial loop over all blocks.
template <int NT>
__device__ __forceinline__ void reduce_partials(const double* mpart, unsigned nblocks, double& a, double& b,
                                                double* sh) {
  a = 0.0;
  b = 0.0;
  // L2 loads (not L1, which is not coherent across SMs), several in flight
#pragma unroll 4
  for (unsigned k = threadIdx.x; k < nblocks; k += NT) { a += __ldcg(mpart + 2 * k); b += __ldcg(mpart + 2 * k + 1); }
  block_sum2<NT>(a, b, sh);
}

// ---- kernels -------------------------------------------------------------

constexpr int kThreads = 256;       // block size of the one-off kernels (state upload, projection)
constexpr int kThreadsStep = 128;   // the step's two kernels on large grids (measured best on GB300)
constexpr int kThreadsNarrow = 32;  // on small grids: one warp per block spreads the FP64 work over more SMs
// Occupancy hint of the interface kernel: at 128 threads, 4 blocks per SM
// (the unconstrained 114 registers, 16 warps) measured 1.4 % faster than 5
// blocks (<= 102 registers, which spill 80 bytes a thread); 6 blocks (80
// registers) spilled more and lost 7 %.
template <int NT> struct iface_min_blocks { static constexpr int value = NT == 128 ? 4 : 1; };

// Blocks of interface_kernel<T, NT> and cell_kernel<T, NT> for a grid.
inline long long iface_blocks(const DevParams& P, int nt) {
  return (P.nfx + nt - 1) / nt + (P.nfy + nt - 1) / nt;
}
inline long long cell_blocks(const DevParams& P, int nt) { return ((long long)P.nx * P.ny + nt - 1) / nt; }

// Load the projected cell at ext index e in the x (ydir = false) or y frame.
template <typename T>
__device__ __forceinline__ Cell<T> load_cell(const DevState<T>& S, long long e, bool ydir) {
  Cell<T> c;
  c.H = S.h[e];
  c.Z = S.z[e];
  c.tau = S.tau[e];
  c.Pi = S.pi[e];
  c.ca = S.ca[e];
  if (!ydir) {
    c.Hn = S.hu[e]; c.Ht = S.hv[e]; c.un = S.u[e]; c.ut = S.v[e]; c.Om = S.omx[e]; c.cb = S.cbx[e];
  } else {
    c.Hn = S.hv[e]; c.Ht = S.hu[e]; c.un = S.v[e]; c.ut = S.u[e]; c.Om = S.omy[e]; c.cb = S.cby[e];
  }
  return c;
}

// One interface of one grid: the x-interface (i - 1/2, j) for k = j (nx + 1)
// + i, or (ydir) the y-interface (i, j - 1/2) for k = j nx + i.  Solves the
// Riemann problem, stores the fluctuations, returns the extreme speed and the
// Newton updates; false if the solve failed (fluctuations zero then).
template <typename T>
__device__ __forceinline__ bool interface_item(const DevParams& P, const DevState<T>& S, bool ydir, long long k,
                                               double& smax, int& iters, int& branch, T* pstar = nullptr) {
  T Am[4], Ap[4], s;
  bool ok;
  if (!ydir) {
    const int row = (int)(k / (P.nx + 1));
    const int i = (int)(k - (long long)row * (P.nx + 1));
    const long long eR = ext_index(P, i, row);
    const Cell<T> L = load_cell(S, eR - 1, false);
    const Cell<T> R = load_cell(S, eR, false);
    ok = riemann_solve(P, L, R, Am, Ap, s, iters, branch, pstar);
#pragma unroll
    for (int c = 0; c < 4; ++c) { S.fx[c * P.nfx + k] = Am[c]; S.fx[(4 + c) * P.nfx + k] = Ap[c]; }
  } else {
    const int row = (int)(k / P.nx);  // j in [0, ny]
    const int i = (int)(k - (long long)row * P.nx);
    const long long eR = ext_index(P, i, row);
    const Cell<T> L = load_cell(S, eR - P.ex, true);
    const Cell<T> R = load_cell(S, eR, true);
    ok = riemann_solve(P, L, R, Am, Ap, s, iters, branch, pstar);
#pragma unroll
    for (int c = 0; c < 4; ++c) { S.fy[c * P.nfy + k] = Am[c]; S.fy[(4 + c) * P.nfy + k] = Ap[c]; }
  }
  smax = (double)s;
  return ok;
}

// Block-wide integer max of non-negative doubles and sum of ints; the
// result is valid in thread 0.
template <int NT>
__device__ __forceinline__ void block_maxbits_sum(double& v, int& n) {
  long long bits = __double_as_longlong(v);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long ob = __shfl_xor_sync(0xffffffffu, bits, o);
    bits = ob > bits ? ob : bits;
    n += __shfl_xor_sync(0xffffffffu, n, o);
  }
  __shared__ long long shb[NT / 32];
  __shared__ int shi[NT / 32];
  if ((threadIdx.x & 31) == 0) { shb[threadIdx.x >> 5] = bits; shi[threadIdx.x >> 5] = n; }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long bb = shb[0];
    int ii = shi[0];
    for (int w = 1; w < NT / 32; ++w) { bb = shb[w] > bb ? shb[w] : bb; ii += shi[w]; }
    v = __longlong_as_double(bb);
    n = ii;
  }
  __syncthreads();
}

// One thread per interface, NT threads per block.  Blocks [0, nbx) cover the
// x-interfaces (i - 1/2, j), i in [0, nx], j in [0, ny); blocks [nbx, nbx +
// nby) the y-interfaces (i, j - 1/2), i in [0, nx), j in [0, ny] (nbx, nby =
// the interface counts over NT, rounded up).  The last block to finish turns
// the step's maximal speeds into its time step.
// ROOTS: also keep each interface's Newton root p* and the doublings of a
// its solve made (roots[k], retries[k], k = x-interfaces then y-interfaces;
// p* = 0 for identical neighbours), for the adjoint's value pass.
template <typename T, int NT = kThreadsStep, bool ROOTS = false>
__global__ void __launch_bounds__(NT, iface_min_blocks<NT>::value) interface_kernel(DevParams P, DevState<T> S, DevScalars* sc,
                                                       const double* fixed_dts, double* dtlog, int fixed,
                                                       T* roots = nullptr, unsigned char* retries = nullptr) {
  // block tallies: the block's maximal speed (bit pattern) and Newton
  // updates, and how many of its warps have added theirs
  __shared__ unsigned long long s_bits;
  __shared__ unsigned int s_its, s_warps, s_halv, s_raised, s_retry;
  if (threadIdx.x == 0) { s_bits = 0ull; s_its = 0u; s_warps = 0u; s_halv = 0u; s_raised = 0u; s_retry = 0u; }
  __syncthreads();
  const unsigned nbx = (unsigned)((P.nfx + NT - 1) / NT);
  const bool ydir = blockIdx.x >= nbx;
  const long long k = (long long)(ydir ? blockIdx.x - nbx : blockIdx.x) * NT + threadIdx.x;
  double smax = 0.0;
  int iters = 0, branch = 0;
  if (k < (ydir ? P.nfy : P.nfx)) {
    if constexpr (ROOTS) {
      T p = T(0);
      if (!interface_item(P, S, ydir, k, smax, iters, branch, &p)) atomicOr(&sc->status, ST_RIEMANN);
      const long long g = ydir ? P.nfx + k : k;
      roots[g] = p;
      retries[g] = (unsigned char)branch_retries(branch);
    } else {
      if (!interface_item(P, S, ydir, k, smax, iters, branch)) atomicOr(&sc->status, ST_RIEMANN);
    }
  }
  // Max of the (non-negative) speeds and sum of the Newton updates, on
  // integers (off the FP64 pipe): over the warp by shuffles, over the block
  // by shared-memory atomics, with no block barrier -- a warp whose Newton
  // loops ended early retires instead of waiting for the slowest warp.  The
  // last warp of the block folds the block's tallies into the step's running
  // maximum (atomic max on the bit pattern: integer order = IEEE order for
  // non-negative doubles; a max is order-free, so the result does not depend
  // on the order the blocks finish in).
  long long bits = __double_as_longlong(smax);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long ob = __shfl_xor_sync(0xffffffffu, bits, o);
    bits = ob > bits ? ob : bits;
    iters += __shfl_xor_sync(0xffffffffu, iters, o);
  }
  const unsigned wb = __reduce_or_sync(0xffffffffu, (unsigned)branch);
  unsigned wr = 0u, wt = 0u, wh = 0u;
  if (wb) {  // a safeguard was taken in this warp (rare): count them
    wr = __reduce_add_sync(0xffffffffu, branch_raised(branch));
    wt = __reduce_add_sync(0xffffffffu, branch_retries(branch));
    wh = __reduce_add_sync(0xffffffffu, branch_halvings(branch));
  }
  if ((threadIdx.x & 31) != 0) return;
  atomicMax(&s_bits, (unsigned long long)bits);
  atomicAdd(&s_its, (unsigned int)iters);
  if (wb) { atomicAdd(&s_raised, wr); atomicAdd(&s_retry, wt); atomicAdd(&s_halv, wh); }
  __threadfence_block();
  if (atomicAdd(&s_warps, 1u) != NT / 32 - 1) return;
  // last warp of the block
  __threadfence_block();
  const unsigned long long bb = atomicMax(&s_bits, 0ull);
  atomicAdd(&sc->newton_iters, (unsigned long long)atomicAdd(&s_its, 0u));
  const unsigned br = atomicAdd(&s_raised, 0u), bt = atomicAdd(&s_retry, 0u), bh = atomicAdd(&s_halv, 0u);
  if (br) atomicAdd(&sc->raised, (unsigned long long)br);
  if (bt) atomicAdd(&sc->retries, (unsigned long long)bt);
  if (bh) atomicAdd(&sc->halvings, (unsigned long long)bh);
  atomicMax(&sc->smax_bits[ydir ? 1 : 0], bb);
  __threadfence();
  if (atomicAdd(&sc->done_iface, 1u) != gridDim.x - 1) return;
  // last block: take the maxima (and reset them for the next step)
  __threadfence();
  const double sx = __longlong_as_double((long long)atomicExch(&sc->smax_bits[0], 0ull));
  const double sy = __longlong_as_double((long long)atomicExch(&sc->smax_bits[1], 0ull));
  double dt;
  const int cs = sc->call_step;
  if (fixed == DT_FIXED) dt = fixed_dts[cs];
  else if (fixed == DT_SPEEDS_ONLY) dt = 0.0;  // set by the caller from all blocks' speeds
  else if (P.dim == 1) dt = P.cfl * P.dx / sx;
  else dt = P.cfl / (sx / P.dx + sy / P.dy);
  if (fixed != DT_SPEEDS_ONLY && (!(dt > 0.0) || !isfinite(dt))) { atomicOr(&sc->status, ST_DT); dt = 0.0; }
  sc->dt = dt;
  sc->Sx = sx;
  sc->Sy = sy;
  dtlog[cs] = dt;
  sc->done_iface = 0u;
}

// One interior cell k = j nx + i of one grid: Godunov average in
// fluctuation form with step dt, friction, checks, projection of the new
// state and its ghosts.  Returns status bits; (mh, mz) = new (h, z).
// Convective part of the cell update (before friction): s = U - dt/dx (A+
// of the left + A- of the right interface) - dt/dy (same in y).
template <typename T>
__device__ __forceinline__ void convect_cell(const DevParams& P, const DevState<T>& S, int i, int j, long long e,
                                             double dt, T s[4]) {
  const T dtx = T(dt * P.inv_dx);
  const long long kx = (long long)j * (P.nx + 1) + i;
  s[0] = S.h[e]; s[1] = S.hu[e]; s[2] = S.hv[e]; s[3] = S.z[e];
  T ax[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) ax[c] = S.fx[(4 + c) * P.nfx + kx] + S.fx[c * P.nfx + kx + 1];
  if (P.dim == 2) {
    const T dty = T(dt * P.inv_dy);
    const long long ky = (long long)j * P.nx + i;
    T ay[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) ay[c] = S.fy[(4 + c) * P.nfy + ky] + S.fy[c * P.nfy + ky + P.nx];
    // y frame (H, Hv, Hu, Z) back to (H, Hu, Hv, Z)
    s[0] = s[0] - (dtx * ax[0] + dty * ay[0]);
    s[1] = s[1] - (dtx * ax[1] + dty * ay[2]);
    s[2] = s[2] - (dtx * ax[2] + dty * ay[1]);
    s[3] = s[3] - (dtx * ax[3] + dty * ay[3]);
  } else {
    s[0] = s[0] - dtx * ax[0];
    s[1] = s[1] - dtx * ax[1];
    s[3] = s[3] - dtx * ax[3];
  }
}

template <typename T>
__device__ __forceinline__ int cell_item(const DevParams& P, const DevState<T>& S, long long k, double dt,
                                         double& mh, double& mz, const Mirror<T>& out = Mirror<T>{}) {
  const int j = (int)(k / P.nx);
  const int i = (int)(k - (long long)j * P.nx);
  const long long e = ext_index(P, i, j);
  T s[4];
  convect_cell(P, S, i, j, e, dt, s);
  const T tau = tdiv(T(1), s[0]);
  // semi-implicit friction: q <- q / (1 + dt C(h) |q|),
  // C = f / (8 h^2) (Darcy) or g / (K^2 h^(7/3)) (Strickler)
  if (P.friction != 0) {
    const T qn = tsqrt(tfma(s[1], s[1], s[2] * s[2]));
    T C = par<T>(P.fric_c, P.f.fric_c) * (tau * tau);
    if (P.friction == 2) C = C * rcbrt64(s[0]);
    const T rden = tdiv(T(1), T(1) + T(dt) * C * qn);
    s[1] = s[1] * rden;
    s[2] = s[2] * rden;
  }
  int st = 0;
  if (!(finite_bits(s[0]) && finite_bits(s[1]) && finite_bits(s[2]) && finite_bits(s[3]))) st = ST_NAN;
  else if (!positive(s[0])) st = ST_NEG_DEPTH;
  store_cell(P, S, e, s, tau);
  write_ghosts(P, S, i, j, s);
  if (out.h) {
    out.h[k] = s[0];
    out.hu[k] = s[1];
    if (P.dim == 2) out.hv[k] = s[2];
    out.z[k] = s[3];
  }
  mh = (double)s[0];
  mz = (double)s[3];
  return st;
}

// One thread per interior cell (i, j): Godunov average in fluctuation form,
// friction, checks, projection of the new state, ghosts, mass partials.
template <typename T, int NT = kThreadsStep>
__global__ void __launch_bounds__(NT) cell_kernel(DevParams P, DevState<T> S, DevScalars* sc, double* mpart,
                                                   Mirror<T> out) {
  // per-thread (h, z) of the new state, and how many warps have stored theirs
  __shared__ double s_m[2][NT];
  __shared__ unsigned int s_warps;
  if (threadIdx.x == 0) s_warps = 0u;
  __syncthreads();
  const long long k = (long long)blockIdx.x * NT + threadIdx.x;
  const long long ncell = (long long)P.nx * P.ny;
  double mh = 0.0, mz = 0.0;
  if (k < ncell) {
    const int st = cell_item(P, S, k, sc->dt, mh, mz, out);
    if (st) atomicOr(&sc->status, st);
  }
  // The block's mass partial, in a fixed order and with no block barrier:
  // the last warp to store its values (shared-memory ticket) adds all NT
  // (lane l: values l, l + 32, ..., then a shuffle tree) and writes the
  // partial; the step's mass sums are taken from the partials on read-out.
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
  a = warp_sum(a);
  b = warp_sum(b);
  if (lane != 0) return;
  mpart[2 * blockIdx.x] = a;
  mpart[2 * blockIdx.x + 1] = b;
  __threadfence();
  if (atomicAdd(&sc->done_cell, 1u) != gridDim.x - 1) return;
  // last block: the step is complete
  sc->mass_parts = gridDim.x;
  sc->t += sc->dt;
  sc->call_step += 1;
  sc->steps += 1;
  sc->done_cell = 0u;
}


// Initialisation: every padded cell; interior cells are projected from the
// state as stored, ghost cells get their rule from the adjacent / periodic
// partner interior cell.  Also checks the state and reduces the masses.
template <typename T>
__global__ void __launch_bounds__(kThreads) init_kernel(DevParams P, DevState<T> S, DevScalars* sc, double* mpart) {
  __shared__ double sh[2 * (kThreads / 32)];
  __shared__ bool last;
  const long long k = (long long)blockIdx.x * kThreads + threadIdx.x;
  const long long ncell = (long long)P.nx * P.ny;
  double mh = 0.0, mz = 0.0;
  if (k < ncell) {
    const int j = (int)(k / P.nx);
    const int i = (int)(k - (long long)j * P.nx);
    const long long e = ext_index(P, i, j);
    T s[4] = {S.h[e], S.hu[e], P.dim == 2 ? S.hv[e] : T(0), S.z[e]};
    if (!(tfinite(s[0]) && tfinite(s[1]) && tfinite(s[2]) && tfinite(s[3]))) atomicOr(&sc->status, ST_NAN);
    else if (!positive(s[0])) atomicOr(&sc->status, ST_NEG_DEPTH);
    store_cell(P, S, e, s, tdiv(T(1), s[0]));
    write_ghosts(P, S, i, j, s);
    mh = (double)s[0];
    mz = (double)s[3];
  }
  block_sum2<kThreads>(mh, mz, sh);
  if (threadIdx.x == 0) {
    mpart[2 * blockIdx.x] = mh;
    mpart[2 * blockIdx.x + 1] = mz;
    __threadfence();
    const unsigned int ticket = atomicAdd(&sc->done_cell, 1u);
    last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  sc->mass_parts = gridDim.x;
  sc->done_cell = 0u;
}

}  // namespace sve
