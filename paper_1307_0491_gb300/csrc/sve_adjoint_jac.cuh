// sve_adjoint_jac.cuh -- the transposed Jacobian of one interface's
// fluctuations, for the discrete adjoint (sve_adjoint.cu).
//
// The fluctuations (A-, A+) of an interface are a function of its two cells'
// conserved states (H, Hn, Ht, Z) in the interface frame and of the Grass
// constants A_g, m_g, through the projection (Grass law written with pow so
// that m_g carries a derivative), the celerity bounds, the Newton constants,
// the root p* of F(p) = 0 and the fan.  The adjoint needs the product of the
// transposed Jacobian with the cotangents (Ab-, Ab+) of the two cells:
//   interface_vjp   reverse mode, written out by hand stage by stage (one
//                   value pass, one backward sweep; the root enters through
//                   the implicit function theorem: the cotangent of p*,
//                   pbar, becomes Fbar = -pbar / F_p on F at fixed p);
//   jac_pass        forward mode with dual numbers through the same
//                   templates the step uses (two passes of five directions,
//                   given the root and the doublings of a the solve made):
//                   the reference the reverse mode is tested against.
// Branches (max of the celerity bounds, signs of the wave speeds) follow the
// values, as in the step.
#pragma once
#include "sve_device.cuh"
#include "sve_dual.cuh"

namespace sve {

// Projection of a conserved state (H, Hn, Ht, Z) in an interface frame with the
// Grass law written through pow, so that A_g and m_g can carry derivatives.
template <typename T>
__device__ __forceinline__ Cell<T> project_grass(const DevParams& P, T H, T Hn, T Ht, T Z, T A, T m) {
  Cell<T> c;
  c.H = H; c.Hn = Hn; c.Ht = Ht; c.Z = Z;
  c.tau = T(1) / H;
  c.un = Hn * c.tau;
  c.ut = Ht * c.tau;
  const T g = par<T>(P.g, P.f.g);
  c.Pi = T(0.5) * g * H * H;
  const T speed2 = c.un * c.un + c.ut * c.ut;
  T Q, dQ;
  if (speed2 == T(0)) {
    Q = T(0);
    dQ = (m == T(1)) ? A : T(0);
  } else {
    const T sp = tsqrt(speed2);
    const T pm1 = tpow(sp, m - T(1));
    const T second = (m - T(1)) * (c.un * c.un) * tpow(sp, m - T(3));
    Q = A * c.un * pm1;
    dQ = A * (pm1 + second);
  }
  c.Om = Q;
  c.ca = H * tsqrt(g * H);
  c.cb = tsqrt(Hn * Hn + g * H * H * dQ);
  return c;
}

// One Jacobian pass with 5 dual directions: PASS 0 = the left state's four
// components and A_g; PASS 1 = the right state's four and m_g.  out[k]
// (k = 0..7 state components in frame order, 8 = A_g, 9 = m_g) receives
// w * sum_c (muL_c dA-_c/dx_k + muR_c dA+_c/dx_k).
template <int PASS>
__device__ __forceinline__ void jac_pass(const DevParams& P, const double u[8], double A, double m, double pstar,
                                         double Fp, const double muL[4], const double muR[4], double w,
                                         double out[10], int retries = 0) {
  using D = Dual<5>;
  D x[10];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = D(u[k]);
  x[8] = D(A);
  x[9] = D(m);
#pragma unroll
  for (int j = 0; j < 4; ++j) x[PASS * 4 + j].d[j] = 1.0;
  x[8 + PASS].d[4] = 1.0;
  const Cell<D> L = project_grass(P, x[0], x[1], x[2], x[3], x[8], x[9]);
  const Cell<D> R = project_grass(P, x[4], x[5], x[6], x[7], x[8], x[9]);
  D a, b;
  celerities(P, L, R, a, b);
  for (int k = 0; k < retries; ++k) a = D(2.0) * a;  // doublings of the step's solve
  NewtonConst<D> c;
  newton_setup(P, L, R, a, b, c);
  NewtonEval<D> e;
  D p(pstar);
  newton_eval(p, c, L, R, e);  // F and its derivatives at the fixed root
#pragma unroll
  for (int j = 0; j < 5; ++j) p.d[j] = -e.F.d[j] / Fp;  // implicit function theorem
  newton_eval(p, c, L, R, e);
  D Am[4], Ap[4];
  fan_fluctuations(P, L, R, c, e, Am, Ap);
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    double s = 0.0;
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) s += muL[cc] * Am[cc].d[j] + muR[cc] * Ap[cc].d[j];
    out[j < 4 ? PASS * 4 + j : 8 + PASS] = w * s;
  }
}


// ---- reverse mode ---------------------------------------------------------

// Values of the projection of one side kept for its backward sweep.
struct ProjRec {
  double H, Hn, Ht, tau, un, ut, sp, pm1, pm3, dQ, ca, cb;
  bool still;  // |U| = 0
  // 1/cb (0 where cb = 0), 1/|U| (0 where |U| = 0), log |U| (Grass)
  double icb, isp, lsp;
  // Shields-parameter laws: tau* = alpha |U|^2, q*, its first two derivatives
  double s2, alpha, q, dq, ddq;
  bool active;  // |U| > 0 and above the threshold
};

// q*, dq*/dtau* and d2q*/dtau*2 of the Shields-parameter laws (the forms of
// shields_rate); false where q* = 0 (below the threshold).
__device__ __forceinline__ bool shields_rate2(const DevParams& P, double ts, double& q, double& dq, double& ddq) {
  const double tcr = P.tau_cr;
  if (P.bedload == 5) {  // Camenen: 12 ts^1.5 exp(-4.5 tcr / ts)
    if (!(ts > 0.0)) return false;
    const double sts = sqrt(ts), its = 1.0 / ts, isq = 1.0 / sts;
    const double e = exp(-4.5 * tcr * its);
    const double g1 = 1.5 * sts + 4.5 * tcr * isq;  // dq = 12 e g1
    q = 12.0 * ts * sts * e;
    dq = 12.0 * e * g1;
    ddq = 12.0 * e * (4.5 * tcr * its * its * g1 + 0.75 * isq - 2.25 * tcr * its * isq);
    return true;
  }
  const double x = ts - tcr;
  if (!(x > 0.0)) return false;
  switch (P.bedload) {
    case 1:    // Meyer-Peter & Mueller: 8 x^1.5
    case 2: {  // Fernandez Luque & Van Beek: 5.7 x^1.5
      const double c = P.bedload == 1 ? 8.0 : 5.7;
      const double sx = sqrt(x);
      q = c * x * sx;
      dq = 1.5 * c * sx;
      ddq = 0.75 * c / sx;
      return true;
    }
    case 3: {  // Nielsen: 12 sqrt(ts) x
      const double sts = sqrt(ts), isq = 1.0 / sts;
      q = 12.0 * sts * x;
      dq = 12.0 * (0.5 * x * isq + sts);
      ddq = 12.0 * (isq - 0.25 * x * isq / ts);
      return true;
    }
    case 4: {  // Ribberink: 11 x^1.65
      q = 11.0 * pow(x, 1.65);
      dq = 1.65 * q / x;
      ddq = 0.65 * dq / x;
      return true;
    }
    default: return false;
  }
}

// Omega = Q and dQ/dun of a Shields-parameter law for the normal velocity un
// and the tangential ut, from the record (as project_shields_rec computes it).
__device__ __forceinline__ void shields_q(const DevParams& P, const ProjRec& r, double un, double ut, double& Q,
                                          double& dQ) {
  Q = 0.0;
  dQ = 0.0;
  if (r.active) {
    const double C = P.qs_scale;
    Q = C * r.q * (un * r.isp);
    dQ = C * (2.0 * r.dq * r.alpha * (un * un) * r.isp + r.q * (ut * ut) * (r.isp * r.isp * r.isp));
  }
}

// Projection of one side with a Shields-parameter law (as closure() in the
// interface frame), keeping its record.
__device__ __forceinline__ Cell<double> project_shields_rec(const DevParams& P, double H, double Hn, double Ht,
                                                            double Z, ProjRec& r) {
  Cell<double> c;
  c.H = H; c.Hn = Hn; c.Ht = Ht; c.Z = Z;
  c.tau = 1.0 / H;
  c.un = Hn * c.tau;
  c.ut = Ht * c.tau;
  c.Pi = 0.5 * P.g * H * H;
  r.s2 = c.un * c.un + c.ut * c.ut;
  r.alpha = P.mpm_alpha;
  if (P.friction != 1) r.alpha = r.alpha * rcbrt64(H);  // Manning: tau* over h^(1/3)
  r.active = r.s2 > 0.0 && shields_rate2(P, r.alpha * r.s2, r.q, r.dq, r.ddq);
  if (r.active) r.isp = 1.0 / sqrt(r.s2);
  double Q, dQ;
  shields_q(P, r, c.un, c.ut, Q, dQ);
  c.Om = Q;
  c.ca = H * sqrt(P.g * H);
  c.cb = sqrt(Hn * Hn + P.g * H * H * dQ);
  r.still = r.s2 == 0.0;
  r.sp = 0.0;
  r.lsp = 0.0;
  r.icb = c.cb > 0.0 ? 1.0 / c.cb : 0.0;
  if (!r.active) r.isp = 0.0;
  r.H = H; r.Hn = Hn; r.Ht = Ht; r.tau = c.tau; r.un = c.un; r.ut = c.ut; r.dQ = dQ; r.ca = c.ca; r.cb = c.cb;
  return c;
}

// Cotangents of one side's projected cell.
struct CellBar {
  double H, Hn, Ht, Z, tau, un, ut, Pi, Om, ca, cb;
};

// Omega = Q and dQ/dun of the Grass law for the normal velocity un, from the
// powers of |U| in the record (as project_grass_rec computes them).
__device__ __forceinline__ void grass_q(const ProjRec& r, double un, double A, double m, double& Q, double& dQ) {
  if (r.still) {
    Q = 0.0;
    dQ = (m == 1.0) ? A : 0.0;
  } else {
    Q = A * un * r.pm1;
    dQ = A * (r.pm1 + (m - 1.0) * (un * un) * r.pm3);
  }
}

__device__ __forceinline__ Cell<double> project_grass_rec(const DevParams& P, double H, double Hn, double Ht,
                                                          double Z, double A, double m, ProjRec& r) {
  Cell<double> c;
  c.H = H; c.Hn = Hn; c.Ht = Ht; c.Z = Z;
  c.tau = 1.0 / H;
  c.un = Hn * c.tau;
  c.ut = Ht * c.tau;
  c.Pi = 0.5 * P.g * H * H;
  const double s2 = c.un * c.un + c.ut * c.ut;
  r.still = s2 == 0.0;
  if (r.still) {
    r.sp = r.pm1 = r.pm3 = 0.0;
  } else {
    r.sp = sqrt(s2);
    // |U|^(m-1), |U|^(m-3): products for the integer exponents of the
    // Grass law in use, pow otherwise
    if (m == 3.0) { r.pm1 = s2; r.pm3 = 1.0; }
    else if (m == 2.0) { r.pm1 = r.sp; r.pm3 = 1.0 / r.sp; }
    else if (m == 4.0) { r.pm1 = s2 * r.sp; r.pm3 = r.sp; }
    else if (m == 1.0) { r.pm1 = 1.0; r.pm3 = 1.0 / s2; }
    else { r.pm1 = pow(r.sp, m - 1.0); r.pm3 = pow(r.sp, m - 3.0); }
  }
  double Q, dQ;
  grass_q(r, c.un, A, m, Q, dQ);
  c.Om = Q;
  c.ca = H * sqrt(P.g * H);
  c.cb = sqrt(Hn * Hn + P.g * H * H * dQ);
  r.H = H; r.Hn = Hn; r.Ht = Ht; r.tau = c.tau; r.un = c.un; r.ut = c.ut; r.dQ = dQ; r.ca = c.ca; r.cb = c.cb;
  // the backward sweep's 1/cb, 1/|U| and log |U| (one divide for both
  // reciprocals where both are needed)
  r.icb = r.isp = r.lsp = 0.0;
  if (c.cb > 0.0 && !r.still) {
    const double q = 1.0 / (c.cb * r.sp);
    r.icb = q * r.sp;
    r.isp = q * c.cb;
  } else if (c.cb > 0.0) {
    r.icb = 1.0 / c.cb;
  } else if (!r.still) {
    r.isp = 1.0 / r.sp;
  }
  if (!r.still) r.lsp = log(r.sp);
  return c;
}

// The backward sweep of a projection (project_grass_rec /
// project_shields_rec) in three parts, so that the transport law's part can
// run once per cell for the sum over the cell's interfaces:
//   proj_fold_bar   the fields other than Omega: cb = sqrt(Hn^2 + g H^2 dQ)
//                   (its cotangent passed on to dQ), ca = H sqrt(g H),
//                   Pi = g H^2 / 2 and (un, ut, tau) -> (H, Hn, Ht, Z), into
//                   ub[0..3]; qb += the cotangents of (Omega, dQ);
//   closure_bar     Omega and dQ of the law in the frame of the record ->
//                   un, ut (unb, utb), H (Hb: a Shields law's alpha through
//                   h^(-1/3) for Strickler) and the parameters (Ab, mb: A_g,
//                   m_g of the Grass law; Kb: the friction coefficient in a
//                   Shields law's tau*);
//   vel_fold_bar    un = Hn tau, ut = Ht tau, tau = 1/H.
__device__ __forceinline__ void vel_fold_bar(const ProjRec& r, double unb, double utb, double taub, double& Hb,
                                             double& Hnb, double& Htb) {
  Hnb += unb * r.tau;
  taub += unb * r.Hn;
  Htb += utb * r.tau;
  taub += utb * r.Ht;
  Hb -= taub * r.tau * r.tau;
}

__device__ __forceinline__ void proj_fold_bar(const DevParams& P, const ProjRec& r, const CellBar& cb, double ub[4],
                                              double qb[2]) {
  double Hb = cb.H, Hnb = cb.Hn, Htb = cb.Ht;
  double dQb = 0.0;
  if (r.cb > 0.0) {
    const double Xb = cb.cb * 0.5 * r.icb;
    Hnb += Xb * 2.0 * r.Hn;
    Hb += Xb * 2.0 * P.g * r.H * r.dQ;
    dQb = Xb * P.g * r.H * r.H;
  }
  Hb += cb.ca * 1.5 * r.ca * r.tau;
  Hb += cb.Pi * P.g * r.H;
  vel_fold_bar(r, cb.un, cb.ut, cb.tau, Hb, Hnb, Htb);
  ub[0] += Hb;
  ub[1] += Hnb;
  ub[2] += Htb;
  ub[3] += cb.Z;
  qb[0] += cb.Om;
  qb[1] += dQb;
}

template <bool GRASS>
__device__ __forceinline__ void closure_bar(const DevParams& P, const ProjRec& r, double A, double m, double Qb,
                                            double dQb, double& unb, double& utb, double& Hb, double& Ab,
                                            double& mb, double& Kb) {
  if constexpr (GRASS) {
    // Om = Q = A un |U|^(m-1); dQ = A (|U|^(m-1) + (m-1) un^2 |U|^(m-3))
    if (r.still) {
      if (m == 1.0) Ab += dQb;
      return;
    }
    const double un2 = r.un * r.un;
    const double second = (m - 1.0) * un2 * r.pm3;
    Ab += Qb * r.un * r.pm1 + dQb * (r.pm1 + second);
    unb += Qb * A * r.pm1;
    const double pm1b = Qb * A * r.un + dQb * A;
    const double secondb = dQb * A;
    mb += secondb * un2 * r.pm3;
    unb += secondb * (m - 1.0) * 2.0 * r.un * r.pm3;
    const double pm3b = secondb * (m - 1.0) * un2;
    const double spb = (pm1b * (m - 1.0) * r.pm1 + pm3b * (m - 3.0) * r.pm3) * r.isp;
    mb += (pm1b * r.pm1 + pm3b * r.pm3) * r.lsp;
    const double s2b = spb * 0.5 * r.isp;
    unb += s2b * 2.0 * r.un;
    utb += s2b * 2.0 * r.ut;
  } else {
    if (!r.active) return;
    // Q = C q un isp, dQ = C (2 dq alpha un^2 isp + q ut^2 isp^3),
    // q = q*(ts), dq = dq*/dts(ts), ts = alpha s2, isp = s2^(-1/2)
    const double C = P.qs_scale, isp = r.isp, isp3 = isp * isp * isp;
    const double un = r.un, ut = r.ut;
    double qb = Qb * C * un * isp;
    unb += Qb * C * r.q * isp;
    double ispb = Qb * C * r.q * un;
    const double dqb = dQb * C * 2.0 * r.alpha * un * un * isp;
    double alphab = dQb * C * 2.0 * r.dq * un * un * isp;
    unb += dQb * C * 4.0 * r.dq * r.alpha * un * isp;
    ispb += dQb * C * (2.0 * r.dq * r.alpha * un * un + 3.0 * r.q * ut * ut * isp * isp);
    qb += dQb * C * ut * ut * isp3;
    utb += dQb * C * 2.0 * r.q * ut * isp3;
    const double tsb = qb * r.dq + dqb * r.ddq;
    alphab += tsb * r.s2;
    const double s2b = tsb * r.alpha - 0.5 * ispb * isp3;
    unb += 2.0 * un * s2b;
    utb += 2.0 * ut * s2b;
    // alpha = f / (8 g (s-1) d_s) for Darcy, n^2 / ((s-1) d_s) h^(-1/3) with
    // n = 1/K for Strickler
    if (P.friction == 1) {
      Kb += alphab * r.alpha / P.fric_coef;
    } else {
      Kb -= alphab * 2.0 * r.alpha / P.fric_coef;
      Hb -= alphab * r.alpha * r.tau * (1.0 / 3.0);
    }
  }
}

// The whole backward sweep of one side's projection: cotangents of its
// cell's fields -> of (H, Hn, Ht, Z) in ub[0..3] and of the parameters.
template <bool GRASS>
__device__ __forceinline__ void project_bar(const DevParams& P, const ProjRec& r, double A, double m,
                                            const CellBar& cb, double ub[4], double& Ab, double& mb, double& Kb) {
  double qb[2] = {0.0, 0.0};
  proj_fold_bar(P, r, cb, ub, qb);
  double unb = 0.0, utb = 0.0, Hb = 0.0, Hnb = 0.0, Htb = 0.0;
  closure_bar<GRASS>(P, r, A, m, qb[0], qb[1], unb, utb, Hb, Ab, mb, Kb);
  vel_fold_bar(r, unb, utb, 0.0, Hb, Hnb, Htb);
  ub[0] += Hb;
  ub[1] += Hnb;
  ub[2] += Htb;
}

// Cotangents of the Newton constants used by the evaluation and the fan.
struct ConstBar {
  double a, b, K, inv_b, inv_K, D, C0, dZ;
};

// Cotangents of the evaluated states.
struct EvalBar {
  double tau1, tau2, tau3, tau4, u1, u4, lam2, lam4, Zs, F;
};

// Backward sweep of newton_eval at fixed constants: eb -> pbar and the
// cotangents of the constants and of both cells' fields.
__device__ __forceinline__ void newton_eval_bar(const NewtonConst<double>& c, const NewtonEval<double>& e,
                                                double p, const Cell<double>& L, const Cell<double>& R,
                                                EvalBar eb, double& pb, ConstBar& cb, CellBar& Lb, CellBar& Rb) {
  // F = (OmL - OmR) + lam2 zl - lam4 zr
  Lb.Om += eb.F;
  Rb.Om -= eb.F;
  eb.lam2 += eb.F * e.zl;
  eb.lam4 -= eb.F * e.zr;
  double zlb = eb.F * e.lam2, zrb = -eb.F * e.lam4;
  // zl = Zs - ZL, zr = Zs - ZR
  eb.Zs += zlb + zrb;
  Lb.Z -= zlb;
  Rb.Z -= zrb;
  // Zs = ZL + K (tau2^2 - tau1^2)
  Lb.Z += eb.Zs;
  cb.K += eb.Zs * (e.tau2 * e.tau2 - e.tau1 * e.tau1);
  eb.tau2 += eb.Zs * 2.0 * c.K * e.tau2;
  eb.tau1 -= eb.Zs * 2.0 * c.K * e.tau1;
  // lam4 = u4 + b tau4, lam2 = u1 - b tau1
  eb.u4 += eb.lam4;
  cb.b += eb.lam4 * e.tau4 - eb.lam2 * e.tau1;
  eb.tau4 += eb.lam4 * c.b;
  eb.u1 += eb.lam2;
  eb.tau1 -= eb.lam2 * c.b;
  // u4 = uR - a (tau4 - tauR), u1 = uL + a (tau1 - tauL)
  Rb.un += eb.u4;
  cb.a += -eb.u4 * (e.tau4 - R.tau) + eb.u1 * (e.tau1 - L.tau);
  eb.tau4 -= eb.u4 * c.a;
  Rb.tau += eb.u4 * c.a;
  Lb.un += eb.u1;
  eb.tau1 += eb.u1 * c.a;
  Lb.tau -= eb.u1 * c.a;
  // tau1 = (p + mm)/2, tau4 = (p - mm)/2
  pb += 0.5 * (eb.tau1 + eb.tau4);
  const double mmb = 0.5 * (eb.tau1 - eb.tau4);
  // mm = -N ip inv_K, ip = 1/p, N = dZ + K D sigma
  const double N = c.dZ + c.K * c.D * (e.tau2 + e.tau3);
  const double Nb = -mmb * e.ip * c.inv_K;
  const double ipb = -mmb * N * c.inv_K;
  cb.inv_K -= mmb * N * e.ip;
  pb -= ipb * e.ip * e.ip;
  const double sigma = e.tau2 + e.tau3;
  cb.dZ += Nb;
  cb.K += Nb * c.D * sigma;
  cb.D += Nb * c.K * sigma;
  double sigmab = Nb * c.K * c.D;
  // tau2 = (sigma - D)/2, tau3 = (sigma + D)/2
  sigmab += 0.5 * (eb.tau2 + eb.tau3);
  cb.D += 0.5 * (eb.tau3 - eb.tau2);
  // sigma = (C0 - (a - b) p) inv_b
  cb.C0 += sigmab * c.inv_b;
  cb.a -= sigmab * p * c.inv_b;
  cb.b += sigmab * p * c.inv_b;
  pb -= sigmab * (c.a - c.b) * c.inv_b;
  cb.inv_b += sigmab * (c.C0 - (c.a - c.b) * p);
}

// Product of the transposed Jacobian of one interface's fluctuations with
// the cotangents Amb (of A-) and Apb (of A+), added to ub[0..7] (left then
// right state, frame order), Ab, mb (A_g, m_g), from the projected cells L, R
// and their records rL, rR (project_grass_rec / project_shields_rec, or the
// same values computed once per cell).  With qb given, the transport law's
// part of both projections' backward sweeps is left out: qb[0..3] receives
// the cotangents of (Omega, dQ) of the left then the right cell (closure_bar
// and vel_fold_bar take them on), and Ab, mb, Kb are not touched.  The value
// pass solves for the root
// as the step does (false if it fails), or, given the root p_root > 0 and the
// doublings of a (retries_in) that the forward solve of this interface at
// this state kept, evaluates the states and F' there once instead of
// iterating.  GRASS: the Grass law (else a Shields-parameter law), compiled
// separately to keep each form's registers.
template <bool GRASS = true>
__device__ __forceinline__ bool interface_vjp_cells(const DevParams& P, const Cell<double>& L,
                                                    const Cell<double>& R, const ProjRec& rL, const ProjRec& rR,
                                                    double A, double m, const double Amb[4], const double Apb[4],
                                                    double ub[8], double& Ab, double& mb, double& Kb,
                                                    double p_root = 0.0, int retries_in = 0,
                                                    double* qb = nullptr) {
  // ---- value pass
  const double g = P.g;
  // celerities (as celerities(), keeping the branches)
  const bool a0L = L.ca >= R.ca, b0L = L.cb >= R.cb;
  const double a0 = a0L ? L.ca : R.ca, b0 = b0L ? L.cb : R.cb;
  const bool aIsA0 = a0 >= b0;
  double a = P.kappa_a * (aIsA0 ? a0 : b0);
  const bool bIsB0 = b0 >= P.beta_min * a0;
  const double b = bIsB0 ? b0 : P.beta_min * a0;
  const bool hL = L.H >= R.H;
  const double Hmax = hL ? L.H : R.H;
  const double dZ = R.Z - L.Z;
  const double adZ = dZ < 0.0 ? -dZ : dZ;
  const double need = b * b + 2.0 * g * P.gamma_z * adZ * (Hmax * Hmax);
  const bool step = a * a < need;
  if (step) a = sqrt(need);
  // the root as the step finds it: the same iterates, and a doubled where
  // the celerities admit no root with positive tau_k (riemann_retry)
  NewtonConst<double> c;
  double pstar;
  NewtonEval<double> e;
  int retries = 0;
  double Fp;
  if (p_root > 0.0) {
    // the forward solve's root: the states and F' there, one evaluation
    retries = retries_in;
    for (int k = 0; k < retries; ++k) a = 2.0 * a;
    newton_setup(P, L, R, a, b, c);
    pstar = p_root;
    newton_eval(pstar, c, L, R, e);
    Fp = newton_deriv(c, e);
  } else {
    for (;; ++retries) {
      double ip0;
      pstar = newton_setup(P, L, R, a, b, c, &ip0);
      newton_eval_ip(pstar, ip0, c, L, R, e);
      int its = 0;
      if (newton_loop(c, L, R, pstar, e, P.newton_maxit, fmax(P.newton_tol, 16.0 * 2.220446049250313e-16), its) &&
          newton_positive(e))
        break;
      if (retries == kARetries) return false;
      a = 2.0 * a;
    }
    Fp = newton_deriv(c, e);
    newton_eval(pstar, c, L, R, e);  // the states at the root, by a full evaluation
  }
  newton_fill(c, L, e);
  // fan (as fan_fluctuations, keeping the branches)
  const double lam1 = L.un - a * L.tau, lam5 = R.un + a * R.tau;
  const double us = e.u1 + b * (e.tau2 - e.tau1);
  const int mi = fan_state(negative(lam1), negative(e.lam2), negative(us), negative(e.lam4), negative(lam5));
  const double a2 = a * a;
  const bool left = mi <= 2;
  const double tk = mi == 1 ? e.tau1 : (mi == 2 ? e.tau2 : (mi == 3 ? e.tau3 : e.tau4));
  const double uk = mi == 1 ? e.u1 : (mi == 4 ? e.u4 : us);
  const double vk = left ? L.ut : R.ut;
  const double zj2 = e.zl, zj4 = -e.zr;  // Z* - ZL, ZR - Z*
  const double d12 = e.tau1 + e.tau2, d34 = e.tau3 + e.tau4;
  // one divide for 1/F_p, 1/tau_k, 1/(tau1 + tau2) and 1/(tau3 + tau4)
  const double t1234 = tk * (d12 * d34);
  const double rr = 1.0 / (Fp * t1234);
  const double iFp = rr * t1234, rt = rr * Fp;
  const double Hk = rt * (d12 * d34);
  const double r12 = rt * (tk * d34), r34 = rt * (tk * d12);
  const double Fh = Hk * uk;
  const double S2 = 2.0 * g * zj2 * r12, S4 = 2.0 * g * zj4 * r34;
  const bool n2 = negative(e.lam2), n4 = negative(e.lam4);

  // ---- backward sweep
  CellBar Lb = {}, Rb = {};
  ConstBar cb = {};
  EvalBar eb = {};
  double ab = 0.0, bb = 0.0;
  // fluctuations
  const double Fhb = Amb[0] - Apb[0], Fqb = Amb[1] - Apb[1], Fvb = Amb[2] - Apb[2];
  // FhX = X.Hn, FqX = X.Hn X.un + X.Pi, FvX = X.Hn X.ut
  double FhLb = -Amb[0], FqLb = -Amb[1], FvLb = -Amb[2];
  double FhRb = Apb[0], FqRb = Apb[1], FvRb = Apb[2];
  const double S2b = n2 ? Amb[1] : Apb[1], S4b = n4 ? Amb[1] : Apb[1];
  const double P2b = n2 ? Amb[3] : Apb[3], P4b = n4 ? Amb[3] : Apb[3];
  eb.lam2 += P2b * zj2;
  eb.lam4 += P4b * zj4;
  double zj2b = P2b * e.lam2 + S2b * 2.0 * g * r12;
  double zj4b = P4b * e.lam4 + S4b * 2.0 * g * r34;
  const double d12b = -S2b * S2 * r12, d34b = -S4b * S4 * r34;
  eb.tau1 += d12b;
  eb.tau2 += d12b;
  eb.tau3 += d34b;
  eb.tau4 += d34b;
  eb.Zs += zj2b - zj4b;
  Lb.Z -= zj2b;
  Rb.Z += zj4b;
  // the flux at x/t = 0: state mi
  if (mi == 0) {
    FhLb += Fhb; FqLb += Fqb; FvLb += Fvb;
  } else if (mi == 5) {
    FhRb += Fhb; FqRb += Fqb; FvRb += Fvb;
  } else {
    // Fv = Fh vk, Fq = Fh uk + Pk, Fh = Hk uk, Hk = 1/tk,
    // Pk = X.Pi + a^2 (X.tau - tk)
    double Fhb2 = Fhb + Fvb * vk + Fqb * uk;
    const double vkb = Fvb * Fh;
    double ukb = Fqb * Fh + Fhb2 * Hk;
    const double Hkb = Fhb2 * uk;
    const double Pkb = Fqb;
    double tkb = -Hkb * Hk * Hk - Pkb * a2;
    CellBar& X = left ? Lb : Rb;
    const Cell<double>& Xc = left ? L : R;
    X.Pi += Pkb;
    X.tau += Pkb * a2;
    ab += 2.0 * a * Pkb * (Xc.tau - tk);
    X.ut += vkb;
    if (mi == 1) eb.u1 += ukb;
    else if (mi == 4) eb.u4 += ukb;
    else {  // us = u1 + b (tau2 - tau1)
      eb.u1 += ukb;
      bb += ukb * (e.tau2 - e.tau1);
      eb.tau2 += ukb * b;
      eb.tau1 -= ukb * b;
    }
    if (mi == 1) eb.tau1 += tkb;
    else if (mi == 2) eb.tau2 += tkb;
    else if (mi == 3) eb.tau3 += tkb;
    else eb.tau4 += tkb;
  }
  Lb.Hn += FhLb + FqLb * L.un + FvLb * L.ut;
  Lb.un += FqLb * L.Hn;
  Lb.Pi += FqLb;
  Lb.ut += FvLb * L.Hn;
  Rb.Hn += FhRb + FqRb * R.un + FvRb * R.ut;
  Rb.un += FqRb * R.Hn;
  Rb.Pi += FqRb;
  Rb.ut += FvRb * R.Hn;
  // the evaluation at p*, directly and through the root (implicit function
  // theorem: Fbar = -pbar / F_p at fixed p), in one backward sweep: the
  // direct cotangent of p, pbar, is the cotangents of the evaluated states
  // against their derivatives in p (those of newton_deriv), so Fbar is known
  // before the sweep, and the sweep is linear in its cotangents
  {
    const double dm = -c.dN * e.ip * c.inv_K - e.m * e.ip;
    const double dt1 = 0.5 + 0.5 * dm, dt4 = 0.5 - 0.5 * dm, dt2 = 0.5 * c.dsig;  // dtau3 = dtau2
    const double dZs = 2.0 * c.K * (e.tau2 * dt2 - e.tau1 * dt1);
    // u1 = uL + a (tau1 - tauL), u4 = uR - a (tau4 - tauR), lam2 = u1 - b tau1,
    // lam4 = u4 + b tau4
    const double pbd = (eb.tau1 + c.a * eb.u1 + c.amb * eb.lam2) * dt1 + (eb.tau2 + eb.tau3) * dt2 +
                       (eb.tau4 - c.a * eb.u4 - c.amb * eb.lam4) * dt4 + eb.Zs * dZs;
    eb.F = -pbd * iFp;
  }
  double pb_unused = 0.0;
  newton_eval_bar(c, e, pstar, L, R, eb, pb_unused, cb, Lb, Rb);
  // Newton constants: a, b, K = (a^2 - b^2)/(2g), inv_b = 1/b,
  // inv_K = 2g/(a^2 - b^2), D = dtau + dPi/a^2, C0 = du + a (tauL + tauR), dZ
  ab += cb.a;
  bb += cb.b;
  const double ig = 2.0 * P.inv_2g;
  ab += cb.K * a * ig;
  bb -= cb.K * b * ig;
  bb -= cb.inv_b * (c.inv_b * c.inv_b);
  ab -= cb.inv_K * c.inv_K * c.inv_K * a * ig;
  bb += cb.inv_K * c.inv_K * c.inv_K * b * ig;
  Rb.tau += cb.D;
  Lb.tau -= cb.D;
  const double ia2 = c.inv_a * c.inv_a;
  Rb.Pi += cb.D * ia2;
  Lb.Pi -= cb.D * ia2;
  ab -= cb.D * (R.Pi - L.Pi) * 2.0 * ia2 * c.inv_a;
  Rb.un += cb.C0;
  Lb.un -= cb.C0;
  ab += cb.C0 * (L.tau + R.tau);
  Lb.tau += cb.C0 * a;
  Rb.tau += cb.C0 * a;
  Rb.Z += cb.dZ;
  Lb.Z -= cb.dZ;
  // a = 2^retries times the celerity of the bounds: back to the latter
  const double a_scale = (double)(1 << retries);
  ab *= a_scale;
  const double inv_a_bound = c.inv_a * a_scale;
  // celerities, along the branches taken
  double a0b = 0.0, b0b = 0.0;
  if (step) {
    const double needb = ab * 0.5 * inv_a_bound;
    bb += needb * 2.0 * b;
    const double sgn = dZ < 0.0 ? -1.0 : 1.0;
    const double dZb = needb * 2.0 * g * P.gamma_z * (Hmax * Hmax) * sgn;
    Rb.Z += dZb;
    Lb.Z -= dZb;
    const double Hmb = needb * 2.0 * g * P.gamma_z * adZ * 2.0 * Hmax;
    if (hL) Lb.H += Hmb;
    else Rb.H += Hmb;
  } else {
    if (aIsA0) a0b += P.kappa_a * ab;
    else b0b += P.kappa_a * ab;
  }
  if (bIsB0) b0b += bb;
  else a0b += P.beta_min * bb;
  if (a0L) Lb.ca += a0b;
  else Rb.ca += a0b;
  if (b0L) Lb.cb += b0b;
  else Rb.cb += b0b;
  // projections
  if (qb) {
    // the laws' part of the projections' backward sweeps left to the caller
    proj_fold_bar(P, rL, Lb, ub, qb);
    proj_fold_bar(P, rR, Rb, ub + 4, qb + 2);
  } else {
    project_bar<GRASS>(P, rL, A, m, Lb, ub, Ab, mb, Kb);
    project_bar<GRASS>(P, rR, A, m, Rb, ub + 4, Ab, mb, Kb);
  }
  return true;
}

// The same product from the two cells' conserved states u[0..7] (left then
// right, frame order), each projected here with its record.
template <bool GRASS = true>
__device__ __forceinline__ bool interface_vjp(const DevParams& P, const double u[8], double A, double m,
                                              const double Amb[4], const double Apb[4], double ub[8], double& Ab,
                                              double& mb, double& Kb, double p_root = 0.0, int retries_in = 0) {
  ProjRec rL, rR;
  const Cell<double> L = GRASS ? project_grass_rec(P, u[0], u[1], u[2], u[3], A, m, rL)
                               : project_shields_rec(P, u[0], u[1], u[2], u[3], rL);
  const Cell<double> R = GRASS ? project_grass_rec(P, u[4], u[5], u[6], u[7], A, m, rR)
                               : project_shields_rec(P, u[4], u[5], u[6], u[7], rR);
  return interface_vjp_cells<GRASS>(P, L, R, rL, rR, A, m, Amb, Apb, ub, Ab, mb, Kb, p_root, retries_in);
}

}  // namespace sve
