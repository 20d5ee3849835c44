/*
 * sve_oracle.c -- plain, slow FP64 CPU stepper for the Saint-Venant--Exner
 * relaxation scheme (Audusse, Delestre, Le, Masson-Fauchier, Navaro, Serra,
 * "Parallelization of a relaxation scheme modelling the bedload transport of
 * sediments in shallow water flow", arXiv:1307.0491).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is
 * checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  It shares no code, header, table or
 * constant with the CUDA library, and the CUDA library never calls it.
 *
 * Build: cc -O2 -ffp-contract=off -fPIC -shared -o libsve_oracle.so sve_oracle.c -lm
 * (-ffp-contract=off: every product and sum is rounded separately, so the
 * result is the same on x86-64 and aarch64.)
 *
 * What it computes, in the paper's order (Sec. 3, the procedure stated after
 * the list of relaxation-model properties):
 *   1. equilibrium projection of the auxiliary variables (lambda -> 0 in
 *      Eqs. relaxpi and relaxqs): Pi = g H^2 / 2, Omega = Q_s(H, u);
 *   2. exact solution of the homogeneous relaxation Riemann problem
 *      (Eqs. relaxh--relaxqs without right-hand side) at every interface,
 *      with constant celerities a, b chosen from the bounds of Eq. (ab);
 *   3. the new cell value = mean over the cell of the juxtaposed Riemann
 *      solutions (Godunov averaging), written in fluctuation form.
 * Around this the hot path adds the pieces the paper leaves unstated, each a
 * reading of the text (see the "readings" list at the end of this comment):
 * the CFL time step, semi-implicit friction (S_f laws of Sec. 2), ghost-cell
 * boundary conditions (one ghost layer, Sec. 4) and mass diagnostics.
 *
 * Riemann solver (derived here from Eqs. relaxh--relaxqs; the paper defers
 * the formulas to its reference [Audusse12]).  With tau = 1/H the five
 * fields are linearly degenerate (Sec. 3, third property of the relaxation
 * model) with speeds
 *     lambda1 = u - a tau,  lambda2 = u - b tau,  lambda3 = u,
 *     lambda4 = u + b tau,  lambda5 = u + a tau.
 * Riemann invariants:
 *   across u +- a tau : u +- a tau, Pi + a^2 tau, Z, Omega
 *   across u +- b tau : u +- b tau, Pi + a^2 tau, Z - K tau^2,
 *                       Omega - lambda Z,        K = (a^2 - b^2) / (2 g)
 *   across u          : u, Pi, Z, Omega  (only tau and the tangential
 *                       velocity jump)
 * Writing the four intermediate states W1..W4 with these invariants leaves
 * one scalar unknown p = tau1 + tau4, fixed by continuity of Omega across
 * the contact; it is found by a safeguarded Newton iteration started from
 * the root of the fluid part alone, p0 = tauL + tauR + (uR - uL)/a.
 *
 * Readings adopted where the paper is silent (each is a choice of this
 * implementation, stated once here):
 *   R1  a = max(kappa_a * max(a0, b0), sqrt(b^2 + 2 g gamma_z |dZ| Hmax^2)),
 *       b = max(b0, beta_min * a0), where a0 = max_{L,R} H sqrt(g H) and
 *       b0 = max_{L,R} sqrt((H u)^2 + g H^2 dQ_s/du) are the lower bounds of
 *       Eq. (ab) (kappa_a > 1 makes a > b so K > 0; the gamma_z term keeps
 *       K tau_min^2 >= gamma_z |dZ|, without which steep bed steps in
 *       near-critical flow have no solution with positive tau_k).
 *   R2  Newton from p0 = tauL + tauR + (uR - uL)/a (the Suliciu root; it
 *       equals the exact root for equal states and for A_g = 0 on a flat
 *       bed, and it is the root continuously connected to the solution
 *       without sediment); stops after the update with |dp| <= newton_tol * p
 *       (default 1e-9: quadratic convergence, with |F''/2F'| p about 25 on
 *       smooth data, leaves an error near 2.5e-17 p, below FP64 rounding);
 *       at most newton_maxit iterations; a step that would make any
 *       tau_k <= 0 (equivalently, break the wave order) is halved, at most
 *       60 times.
 *   R3  Bitwise-identical left and right states give zero fluctuations
 *       without a solve.
 *   R4  2D: unsplit method of lines (Sec. 4) -- x and y fluctuations of the
 *       same state n enter one forward-Euler update; the tangential velocity
 *       is passive and jumps only at the contact.
 *   R5  CFL: dt = cfl * dx / Sx (1D), dt = cfl / (Sx/dx + Sy/dy) (2D), S the
 *       max over interfaces of max(|lambda1|, |lambda5|).
 *   R6  Friction after the convective update, semi-implicit:
 *       q <- q / (1 + dt C(h) |q|), C = f/(8 h^2) (Darcy-Weisbach) or
 *       g/(K^2 h^(7/3)) (Strickler, n = 1/K), from S_f in Sec. 2.
 *   R7  Ghost cells: PERIODIC wrap; FREE copies the adjacent cell; INFLOW_Q
 *       copies h and z_b and sets the inward normal discharge q_in;
 *       INFLOW_QH also sets h = h_in; WALL mirrors (normal discharge
 *       negated).  Ghost Pi and Omega are projected from the ghost state.
 *   R8  Meyer-Peter & Mueller (Eq. MPM): q_b = sqrt((s-1) g d_s^3) *
 *       8 (tau* - tau*_cr)_+^(3/2) in the direction of the velocity, with
 *       tau* from the friction law: f |U|^2 / (8 g (s-1) d_s) (Darcy) or
 *       n^2 |U|^2 / ((s-1) d_s h^(1/3)) (Manning).  The other laws of the
 *       list in Sec. 2 (Eqs. FLVB, Nielsen, Ribberink, Camenen) replace the
 *       non-dimensional rate q* in the same way.
 *   R13 The splitting scheme (orc_split_run, the alternative Sec. 2
 *       contrasts with the coupled method): the step with the transport
 *       switched off for (h, hu, hv) over the fixed bed, then a first-order
 *       Exner update of the bed with the bedload flux upwinded by the sign of
 *       the interfaces' mean normal velocity.
 */
#include <math.h>
#include <stddef.h>
#include <string.h>
#include <stdlib.h>

/* ---- parameters (own definition; mirrors nothing) ---------------------- */
/* transport laws of Sec. 2: Grass, then the Shields-parameter laws of
 * Eqs. MPM, FLVB, Nielsen, Ribberink, Camenen */
enum { ORC_GRASS = 0, ORC_MPM = 1, ORC_FLVB = 2, ORC_NIELSEN = 3, ORC_RIBBERINK = 4, ORC_CAMENEN = 5 };
enum { ORC_FRIC_NONE = 0, ORC_FRIC_DARCY = 1, ORC_FRIC_STRICKLER = 2 };
enum { ORC_BC_PERIODIC = 0, ORC_BC_FREE = 1, ORC_BC_INFLOW_Q = 2, ORC_BC_INFLOW_QH = 3, ORC_BC_WALL = 4 };
enum {
  ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_NEG_DEPTH = -4, ORC_ERR_RIEMANN = -5, ORC_ERR_NAN = -6, ORC_ERR_DT = -7
};

typedef struct {
  int dim, nx, ny;
  double lx, ly, g, cfl;
  int bedload;
  double A_g, m_g;
  double s, d_s, tau_cr;
  int friction;
  double f_dw, K_st;
  int bc[4]; /* W, E, S, N */
  double q_in, h_in;
  double kappa_a, beta_min, gamma_z;
  double newton_tol;
  int newton_maxit;
} orc_params;

typedef struct {
  double a, b, K;
  double lam[5];
  /* states L, W1, W2, W3, W4, R */
  double tau[6], u[6], v[6], Z[6], Pi[6], Om[6];
  double Am[4], Ap[4]; /* fluctuations of (H, H u_n, H u_t, Z) */
  int iters, status;
  /* which safeguards this solve used: halvings = Newton steps halved (summed
   * over the accepted updates and the attempts); raised = 1 if the bed-jump
   * bound of reading R1 set a; retries = how often a was doubled (reading
   * R12) -- counters for the tests, no effect on the result */
  int halvings, raised, retries;
} orc_riemann_out;

/* ---- closures (Sec. 2) ------------------------------------------------- */

/* |U|^k for integer k >= 0 by repeated multiplication, otherwise pow. */
static double orc_speed_pow(double speed2, double speed, double k) {
  if (k == 0.0) return 1.0;
  if (k == 1.0) return speed;
  if (k == 2.0) return speed2;
  if (k == 3.0) return speed2 * speed;
  return pow(speed, k);
}

/* Non-dimensional transport rate q*_b(tau*) of the laws listed in Sec. 2 and
 * its derivative dq*_b/dtau*; tcr = tau*_cr.  (x)_+ = max(x, 0).
 *   MPM (Eq. MPM):          q* = 8   (tau* - tcr)_+^(3/2)
 *   FLvB (Eq. FLVB):        q* = 5.7 (tau* - tcr)_+^(3/2)
 *   Nielsen (Eq. Nielsen):  q* = 12 sqrt(tau*) (tau* - tcr)_+
 *   Ribberink (Eq. Ribberink): q* = 11 (tau* - tcr)_+^1.65
 *   Camenen (Eq. Camenen):  q* = 12 tau*^(3/2) exp(-4.5 tcr / tau*)
 * (no threshold; 0 at tau* = 0). */
static void orc_qstar(int law, double ts, double tcr, double* q, double* dq) {
  *q = 0.0;
  *dq = 0.0;
  if (law == ORC_CAMENEN) {
    if (ts <= 0.0) return;
    double e = exp(-4.5 * tcr / ts);
    *q = 12.0 * ts * sqrt(ts) * e;
    /* d/dts: 12 e [1.5 sqrt(ts) + ts^(3/2) 4.5 tcr / ts^2] */
    *dq = 12.0 * e * (1.5 * sqrt(ts) + 4.5 * tcr / sqrt(ts));
    return;
  }
  double x = ts - tcr;
  if (x <= 0.0) return;
  switch (law) {
    case ORC_MPM:
      *q = 8.0 * x * sqrt(x);
      *dq = 8.0 * 1.5 * sqrt(x);
      break;
    case ORC_FLVB:
      *q = 5.7 * x * sqrt(x);
      *dq = 5.7 * 1.5 * sqrt(x);
      break;
    case ORC_NIELSEN:
      *q = 12.0 * sqrt(ts) * x;
      *dq = 12.0 * (x / (2.0 * sqrt(ts)) + sqrt(ts));
      break;
    case ORC_RIBBERINK:
      *q = 11.0 * pow(x, 1.65);
      *dq = 11.0 * 1.65 * pow(x, 0.65);
      break;
    default:
      break;
  }
}

/* Bedload flux normal component Omega = Q_s . n and its derivative with
 * respect to the normal velocity at fixed H (needed by the bound on b in
 * Eq. ab).  un, ut: normal and tangential velocity.
 *   Grass (Eq. bedload Grass, 2D form q_b = A_g U |U|^(m_g-1)):
 *     Q = A_g un |U|^(m-1),  dQ/dun = A_g (|U|^(m-1) + (m-1) un^2 |U|^(m-3))
 *   Shields-parameter laws (Eqs. MPM, FLVB, Nielsen, Ribberink, Camenen
 *     with the non-dimensional form of Sec. 2), reading R8:
 *     Q = sqrt((s-1) g d_s^3) q*(tau*) un/|U|, tau* = alpha |U|^2. */
static void orc_closure(const orc_params* P, double H, double un, double ut, double* Q, double* dQ) {
  double speed2 = un * un + ut * ut;
  if (P->bedload == ORC_GRASS) {
    double m = P->m_g;
    if (speed2 == 0.0) {
      *Q = 0.0;
      *dQ = (m == 1.0) ? P->A_g : 0.0;
      return;
    }
    double speed = sqrt(speed2);
    double pm1 = orc_speed_pow(speed2, speed, m - 1.0);
    *Q = P->A_g * un * pm1;
    double second = 0.0;
    if (m != 1.0) {
      /* (m-1) un^2 |U|^(m-3) */
      double pm3 = (m == 3.0) ? 1.0 : ((m == 2.0) ? 1.0 / speed : ((m == 4.0) ? speed : pow(speed, m - 3.0)));
      second = (m - 1.0) * (un * un) * pm3;
    }
    *dQ = P->A_g * (pm1 + second);
    return;
  }
  /* Shields-parameter laws: Q_b = q*(tau*) sqrt((s-1) g d_s^3) along U/|U|,
   * tau* = tau_b / ((rho_s - rho) g d_s) with tau_b = rho g h S_f (Sec. 2),
   * i.e. tau* = alpha |U|^2 for the friction law in use */
  double alpha;
  double sm1 = P->s - 1.0;
  if (P->friction == ORC_FRIC_DARCY) {
    alpha = P->f_dw / (8.0 * P->g * sm1 * P->d_s);
  } else {
    double n = 1.0 / P->K_st;
    alpha = (n * n) / (sm1 * P->d_s * cbrt(H));
  }
  double tstar = alpha * speed2;
  double qs, dqs; /* q* at tau* and its derivative in tau* */
  orc_qstar(P->bedload, tstar, P->tau_cr, &qs, &dqs);
  if (speed2 == 0.0 || (qs == 0.0 && dqs == 0.0)) {
    *Q = 0.0;
    *dQ = 0.0;
    return;
  }
  double speed = sqrt(speed2);
  double Cs = sqrt(sm1 * P->g * P->d_s * P->d_s * P->d_s);
  *Q = Cs * qs * (un / speed);
  /* d/dun [q*(alpha |U|^2) un/|U|] = q*'(tau*) (2 alpha un) un/|U|
   *                                 + q*(tau*) ut^2/|U|^3 */
  double d1 = 2.0 * dqs * alpha * (un * un) / speed;
  double d2 = qs * (ut * ut) / (speed2 * speed);
  *dQ = Cs * (d1 + d2);
}

/* ---- equilibrium projection (lambda -> 0 in Eqs. relaxpi, relaxqs) ---- */
typedef struct {
  double H, tau, un, ut, Z, Pi, Om;
  double ca; /* H sqrt(g H): lower bound on a, Eq. (ab) */
  double cb; /* sqrt((H un)^2 + g H^2 dQ/dun): lower bound on b, Eq. (ab) */
} orc_cell;

static orc_cell orc_project(const orc_params* P, double H, double Hun, double Hut, double Z) {
  orc_cell c;
  c.H = H;
  c.tau = 1.0 / H;
  c.un = Hun / H;
  c.ut = Hut / H;
  c.Z = Z;
  c.Pi = 0.5 * P->g * H * H;
  double Q, dQ;
  orc_closure(P, H, c.un, c.ut, &Q, &dQ);
  c.Om = Q;
  c.ca = H * sqrt(P->g * H);
  c.cb = sqrt(Hun * Hun + P->g * H * H * dQ);
  return c;
}

/* ---- homogeneous relaxation Riemann problem ----------------------------- */

/* Celerities of one interface, reading R1: the lower bounds of Eq. (ab)
 * taken over both states, a scaled by kappa_a, b floored at beta_min a0,
 * and a raised where needed so that K = (a^2 - b^2)/(2g) satisfies
 * K tau_min^2 >= gamma_z |Z_R - Z_L| (the sediment waves can carry the bed
 * jump; one of the "stronger bounds" Sec. 3 says well-definedness may need). */
static int orc_celerities(const orc_params* P, const orc_cell* L, const orc_cell* R, double* a_out,
                          double* b_out) {
  double a0 = L->ca > R->ca ? L->ca : R->ca;
  double b0 = L->cb > R->cb ? L->cb : R->cb;
  double a = P->kappa_a * (a0 > b0 ? a0 : b0);
  double bfloor = P->beta_min * a0;
  double b = b0 > bfloor ? b0 : bfloor;
  double Hmax = L->H > R->H ? L->H : R->H;
  double need = b * b + 2.0 * P->g * P->gamma_z * fabs(R->Z - L->Z) * (Hmax * Hmax);
  int raised = a * a < need;
  if (raised) a = sqrt(need);
  *a_out = a;
  *b_out = b;
  return raised;
}

typedef struct {
  double tau[4], u[4]; /* tau1..tau4, u1, u*, u*, u4 */
  double lam2, lam4, Zs, F, dF;
} orc_eval;

/* Intermediate states as functions of p = tau1 + tau4 (all invariant
 * relations of the a- and b-waves and the contact hold for every p; only the
 * continuity of Omega across the contact, F(p) = 0, remains). */
static void orc_eval_p(double p, double a, double b, double K, double D, double du, double dZ,
                       const orc_cell* L, const orc_cell* R, int want_dF, orc_eval* e) {
  /* u* from the left equals u* from the right  =>  sigma = tau2 + tau3 */
  double sigma = (du + a * (L->tau + R->tau) - (a - b) * p) / b;
  double tau2 = 0.5 * (sigma - D);
  double tau3 = 0.5 * (sigma + D);
  /* Z* from the left equals Z* from the right  =>  m = tau1 - tau4 */
  double N = dZ + K * D * sigma;
  double m = -N / (K * p);
  double tau1 = 0.5 * (p + m);
  double tau4 = 0.5 * (p - m);
  double u1 = L->un + a * (tau1 - L->tau);
  double us = u1 + b * (tau2 - tau1);
  double u4 = R->un - a * (tau4 - R->tau);
  double lam2 = u1 - b * tau1;
  double lam4 = u4 + b * tau4;
  double Zs = L->Z + K * (tau2 * tau2 - tau1 * tau1);
  e->tau[0] = tau1; e->tau[1] = tau2; e->tau[2] = tau3; e->tau[3] = tau4;
  e->u[0] = u1; e->u[1] = us; e->u[2] = us; e->u[3] = u4;
  e->lam2 = lam2;
  e->lam4 = lam4;
  e->Zs = Zs;
  /* Omega continuity across the contact */
  e->F = (L->Om - R->Om) + lam2 * (Zs - L->Z) - lam4 * (Zs - R->Z);
  if (want_dF) {
    double dsigma = -(a - b) / b;
    double dtau2 = 0.5 * dsigma;
    double dN = K * D * dsigma;
    double dm = -dN / (K * p) - m / p;
    double dtau1 = 0.5 * (1.0 + dm);
    double dtau4 = 0.5 * (1.0 - dm);
    double dlam2 = (a - b) * dtau1;
    double dlam4 = -(a - b) * dtau4;
    double dZs = 2.0 * K * (tau2 * dtau2 - tau1 * dtau1);
    e->dF = dlam2 * (Zs - L->Z) + lam2 * dZs - dlam4 * (Zs - R->Z) - lam4 * dZs;
  }
}

static int orc_tau_positive(const orc_eval* e) {
  return e->tau[0] > 0.0 && e->tau[1] > 0.0 && e->tau[2] > 0.0 && e->tau[3] > 0.0;
}

/* The Riemann problem at the celerities (a, b): the scalar Newton iteration
 * in p, then the intermediate states and the fluctuations.  ORC_ERR_RIEMANN
 * if no root with positive tau_k was reached. */
static int orc_solve_at(const orc_params* P, const orc_cell* L, const orc_cell* R, const double Lc[4],
                        const double Rc[4], double a, double b, orc_riemann_out* o) {
  double K = (a * a - b * b) / (2.0 * P->g);
  o->a = a; o->b = b; o->K = K;
  o->lam[0] = L->un - a * L->tau;
  o->lam[4] = R->un + a * R->tau;
  double D = (R->tau - L->tau) + (R->Pi - L->Pi) / (a * a);
  double du = R->un - L->un;
  double dZ = R->Z - L->Z;
  /* reading R2: start from the root of the fluid part alone (the Suliciu
   * solution, where the b-waves carry no jump: tau1 = tau2, tau3 = tau4,
   * so p = sigma); exact for equal states and for A_g = 0 on a flat bed */
  double p = L->tau + R->tau + du / a;
  orc_eval e;
  orc_eval_p(p, a, b, K, D, du, dZ, L, R, 1, &e);
  int converged = 0;
  int it;
  for (it = 1; it <= P->newton_maxit; ++it) {
    double dp = -e.F / e.dF;
    if (!isfinite(dp)) break;
    double step = dp;
    orc_eval trial;
    int ok = 0, halved = 0;
    for (int halve = 0; halve <= 60; ++halve) {
      orc_eval_p(p + step, a, b, K, D, du, dZ, L, R, 1, &trial);
      if (orc_tau_positive(&trial)) { ok = 1; halved = halve; break; }
      step = 0.5 * step;
    }
    if (!ok) break;
    o->halvings += halved;
    p = p + step;
    e = trial;
    /* only a full Newton step measures the distance to the root: a step
     * shortened to keep the tau_k positive is small because the iterate sits
     * at the edge of the admissible set, not because F is small there */
    if (!halved && fabs(step) <= P->newton_tol * p) { converged = 1; break; }
  }
  o->iters += it;
  if (!converged || !orc_tau_positive(&e)) return ORC_ERR_RIEMANN;

  double a2 = a * a;
  /* states L, W1, W2, W3, W4, R in (tau, u, v, Z, Pi, Omega) */
  o->tau[0] = L->tau; o->u[0] = L->un; o->v[0] = L->ut; o->Z[0] = L->Z; o->Pi[0] = L->Pi; o->Om[0] = L->Om;
  o->tau[5] = R->tau; o->u[5] = R->un; o->v[5] = R->ut; o->Z[5] = R->Z; o->Pi[5] = R->Pi; o->Om[5] = R->Om;
  for (int k = 0; k < 4; ++k) { o->tau[k + 1] = e.tau[k]; o->u[k + 1] = e.u[k]; }
  o->v[1] = L->ut; o->v[2] = L->ut; o->v[3] = R->ut; o->v[4] = R->ut;
  o->Z[1] = L->Z; o->Z[2] = e.Zs; o->Z[3] = e.Zs; o->Z[4] = R->Z;
  o->Pi[1] = L->Pi + a2 * (L->tau - e.tau[0]);
  o->Pi[2] = L->Pi + a2 * (L->tau - e.tau[1]);
  o->Pi[3] = R->Pi + a2 * (R->tau - e.tau[2]);
  o->Pi[4] = R->Pi + a2 * (R->tau - e.tau[3]);
  o->Om[1] = L->Om;
  o->Om[2] = L->Om + e.lam2 * (e.Zs - L->Z);
  o->Om[3] = o->Om[2];
  o->Om[4] = R->Om;
  o->lam[1] = e.lam2;
  o->lam[2] = e.u[1];
  o->lam[3] = e.lam4;

  /* conserved states U = (H, H un, H ut, Z) of the six regions */
  double U[6][4];
  for (int c = 0; c < 4; ++c) { U[0][c] = Lc[c]; U[5][c] = Rc[c]; }
  for (int k = 1; k <= 4; ++k) {
    double Hk = 1.0 / o->tau[k];
    U[k][0] = Hk;
    U[k][1] = Hk * o->u[k];
    U[k][2] = Hk * o->v[k];
    U[k][3] = o->Z[k];
  }
  /* fluctuations: A- = sum_{lam<0} lam [U], A+ = sum_{lam>0} lam [U] */
  for (int c = 0; c < 4; ++c) { o->Am[c] = 0.0; o->Ap[c] = 0.0; }
  for (int k = 0; k < 5; ++k) {
    double lk = o->lam[k];
    for (int c = 0; c < 4; ++c) {
      double jump = U[k + 1][c] - U[k][c];
      if (lk < 0.0) o->Am[c] += lk * jump;
      else if (lk > 0.0) o->Ap[c] += lk * jump;
    }
  }
  return ORC_OK;
}

/* Solve one interface.  L, R projected cells; Lc, Rc their conserved states
 * (H, H un, H ut, Z).  Fills o (states, speeds, fluctuations).  Celerities
 * of reading R1; where they admit no solution with positive tau_k, a is
 * doubled and the problem solved again, at most ORC_A_RETRIES times
 * (reading R12). */
#define ORC_A_RETRIES 3
static int orc_solve(const orc_params* P, const orc_cell* L, const orc_cell* R, const double Lc[4],
                     const double Rc[4], orc_riemann_out* o) {
  memset(o, 0, sizeof(*o));
  o->status = ORC_OK;
  double a, b;
  o->raised = orc_celerities(P, L, R, &a, &b);

  /* reading R3: identical states */
  if (Lc[0] == Rc[0] && Lc[1] == Rc[1] && Lc[2] == Rc[2] && Lc[3] == Rc[3]) {
    o->a = a; o->b = b; o->K = (a * a - b * b) / (2.0 * P->g);
    o->lam[0] = L->un - a * L->tau;
    o->lam[1] = L->un - b * L->tau;
    o->lam[2] = L->un;
    o->lam[3] = L->un + b * L->tau;
    o->lam[4] = R->un + a * R->tau;
    for (int k = 0; k < 6; ++k) {
      o->tau[k] = L->tau; o->u[k] = L->un; o->v[k] = L->ut; o->Z[k] = L->Z; o->Pi[k] = L->Pi; o->Om[k] = L->Om;
    }
    return ORC_OK;
  }
  for (;;) {
    if (orc_solve_at(P, L, R, Lc, Rc, a, b, o) == ORC_OK) return ORC_OK;
    if (o->retries == ORC_A_RETRIES) {
      o->status = ORC_ERR_RIEMANN;
      return ORC_ERR_RIEMANN;
    }
    a = 2.0 * a;
    o->retries += 1;
  }
}

/* ---- ghost cells (reading R7) ------------------------------------------ */

/* Ghost value for a boundary cell.  side: 0 W, 1 E, 2 S, 3 N.  in = the
 * adjacent interior (or periodic partner) state (H, Hu, Hv, Z) in x/y
 * components; out = ghost state in the same components. */
static void orc_ghost(const orc_params* P, int side, const double in[4], double out[4]) {
  int type = P->bc[side];
  int normal = (side < 2) ? 1 : 2;   /* index of the normal discharge */
  int tangent = (side < 2) ? 2 : 1;
  double inward = (side == 0 || side == 2) ? 1.0 : -1.0;
  for (int c = 0; c < 4; ++c) out[c] = in[c];
  switch (type) {
    case ORC_BC_PERIODIC:
    case ORC_BC_FREE:
      break;
    case ORC_BC_INFLOW_Q:
      out[normal] = inward * P->q_in;
      out[tangent] = 0.0;
      break;
    case ORC_BC_INFLOW_QH:
      out[0] = P->h_in;
      out[normal] = inward * P->q_in;
      out[tangent] = 0.0;
      break;
    case ORC_BC_WALL:
      out[normal] = -in[normal];
      break;
    default:
      break;
  }
}

/* ---- one time step ------------------------------------------------------ */

static int orc_check_cell(double H, double q1, double q2, double Z) {
  if (!(isfinite(H) && isfinite(q1) && isfinite(q2) && isfinite(Z))) return ORC_ERR_NAN;
  if (!(H > 0.0)) return ORC_ERR_NEG_DEPTH;
  return ORC_OK;
}

/* Friction, reading R6.  h: depth after convection; q1, q2: discharge. */
static void orc_friction(const orc_params* P, double dt, double h, double* q1, double* q2) {
  if (P->friction == ORC_FRIC_NONE) return;
  double qn = sqrt((*q1) * (*q1) + (*q2) * (*q2));
  double C;
  if (P->friction == ORC_FRIC_DARCY) {
    C = P->f_dw / (8.0 * h * h);
  } else {
    double h73 = h * h * cbrt(h);
    C = P->g / (P->K_st * P->K_st * h73);
  }
  double den = 1.0 + dt * C * qn;
  *q1 = *q1 / den;
  *q2 = *q2 / den;
}

/* Extended (ghost-padded) arrays: index (j+1)*(nx+2) + (i+1), i in [-1, nx],
 * j in [-1, ny]; in 1D ny = 1 and only the row j = 0 is used. */
typedef struct {
  int nx, ny, ex;
  double *H, *Hu, *Hv, *Z;
} orc_ext;

static int orc_ext_alloc(orc_ext* X, int nx, int ny) {
  X->nx = nx; X->ny = ny; X->ex = nx + 2;
  size_t n = (size_t)(nx + 2) * (size_t)(ny + 2);
  X->H = calloc(n, sizeof(double));
  X->Hu = calloc(n, sizeof(double));
  X->Hv = calloc(n, sizeof(double));
  X->Z = calloc(n, sizeof(double));
  return (X->H && X->Hu && X->Hv && X->Z) ? ORC_OK : ORC_ERR_ARG;
}
static void orc_ext_free(orc_ext* X) {
  free(X->H); free(X->Hu); free(X->Hv); free(X->Z);
}
static size_t orc_xi(const orc_ext* X, int i, int j) { return (size_t)(j + 1) * X->ex + (size_t)(i + 1); }

static void orc_ext_get(const orc_ext* X, int i, int j, double s[4]) {
  size_t k = orc_xi(X, i, j);
  s[0] = X->H[k]; s[1] = X->Hu[k]; s[2] = X->Hv[k]; s[3] = X->Z[k];
}
static void orc_ext_put(orc_ext* X, int i, int j, const double s[4]) {
  size_t k = orc_xi(X, i, j);
  X->H[k] = s[0]; X->Hu[k] = s[1]; X->Hv[k] = s[2]; X->Z[k] = s[3];
}

/* Fill the padded arrays from the state and apply the ghost rules.  In 1D
 * (dim 1) hv is NULL and only the W/E ghosts exist. */
static void orc_fill(const orc_params* P, orc_ext* X, const double* h, const double* hu, const double* hv,
                     const double* z) {
  int nx = X->nx, ny = X->ny;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t c = (size_t)j * nx + i;
      double s[4] = {h[c], hu[c], hv ? hv[c] : 0.0, z[c]};
      orc_ext_put(X, i, j, s);
    }
  double in[4], out[4];
  for (int j = 0; j < ny; ++j) {
    orc_ext_get(X, P->bc[0] == ORC_BC_PERIODIC ? nx - 1 : 0, j, in);
    orc_ghost(P, 0, in, out);
    orc_ext_put(X, -1, j, out);
    orc_ext_get(X, P->bc[1] == ORC_BC_PERIODIC ? 0 : nx - 1, j, in);
    orc_ghost(P, 1, in, out);
    orc_ext_put(X, nx, j, out);
  }
  if (P->dim == 2) {
    for (int i = 0; i < nx; ++i) {
      orc_ext_get(X, i, P->bc[2] == ORC_BC_PERIODIC ? ny - 1 : 0, in);
      orc_ghost(P, 2, in, out);
      orc_ext_put(X, i, -1, out);
      orc_ext_get(X, i, P->bc[3] == ORC_BC_PERIODIC ? 0 : ny - 1, in);
      orc_ghost(P, 3, in, out);
      orc_ext_put(X, i, ny, out);
    }
  }
}

/* Projection of every cell incl. ghosts, in x-normal orientation (un = u,
 * ut = v).  The y-direction projection is done per interface below. */
static orc_cell orc_project_dir(const orc_params* P, const orc_ext* X, int i, int j, int ydir) {
  size_t k = orc_xi(X, i, j);
  if (!ydir) return orc_project(P, X->H[k], X->Hu[k], X->Hv[k], X->Z[k]);
  return orc_project(P, X->H[k], X->Hv[k], X->Hu[k], X->Z[k]);
}

static void orc_conserved(const orc_ext* X, int i, int j, int ydir, double c[4]) {
  size_t k = orc_xi(X, i, j);
  c[0] = X->H[k];
  c[1] = ydir ? X->Hv[k] : X->Hu[k];
  c[2] = ydir ? X->Hu[k] : X->Hv[k];
  c[3] = X->Z[k];
}

/* Cell sizes of the whole grid (a padded block of a domain decomposition
 * uses the same ones). */
static double orc_dx(const orc_params* P) { return P->lx / P->nx; }
static double orc_dy(const orc_params* P) { return (P->dim == 2) ? P->ly / P->ny : 1.0; }

/* CFL time step from the extreme speeds (reading R5). */
static double orc_dt_of_speeds(const orc_params* P, double Sx, double Sy) {
  if (P->dim == 1) return P->cfl * orc_dx(P) / Sx;
  return P->cfl / (Sx / orc_dx(P) + Sy / orc_dy(P));
}

/* Validity of a padded state (interior and ghosts, corners excepted). */
static int orc_ext_check(const orc_params* P, const orc_ext* X) {
  int nx = X->nx, ny = X->ny;
  for (int j = (P->dim == 2 ? -1 : 0); j <= (P->dim == 2 ? ny : ny - 1); ++j)
    for (int i = -1; i <= nx; ++i) {
      int corner = (P->dim == 2) && (i < 0 || i >= nx) && (j < 0 || j >= ny);
      if (corner) continue;
      size_t k = orc_xi(X, i, j);
      int st = orc_check_cell(X->H[k], X->Hu[k], X->Hv[k], X->Z[k]);
      if (st) return st;
    }
  return ORC_OK;
}

/* The Riemann problems of Sec. 3 on a padded block whose ghosts are
 * filled: one solve per interface; acc[4 c + comp] receives the cell's net
 * fluctuation (A+ of its left / lower interface + A- of its right / upper
 * one, over dx, dy; comp = H, Hu, Hv, Z) and (Sx, Sy) the extreme wave
 * speeds max(|lambda1|, |lambda5|) of the x and y solves (reading R5, with
 * the celerity a each solve used). */
static int orc_ext_solve(const orc_params* P, const orc_ext* X, double* acc /* 4 nx ny */, double* Sx_out,
                         double* Sy_out) {
  int nx = X->nx, ny = X->ny;
  double dx = orc_dx(P);
  double dy = orc_dy(P);
  double Sx = 0.0, Sy = 0.0;
  memset(acc, 0, sizeof(double) * 4 * (size_t)nx * ny);
  orc_riemann_out o;
  /* x-interfaces i - 1/2, i = 0..nx */
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i <= nx; ++i) {
      orc_cell L = orc_project_dir(P, X, i - 1, j, 0);
      orc_cell R = orc_project_dir(P, X, i, j, 0);
      double Lc[4], Rc[4];
      orc_conserved(X, i - 1, j, 0, Lc);
      orc_conserved(X, i, j, 0, Rc);
      int st = orc_solve(P, &L, &R, Lc, Rc, &o);
      if (st) return st;
      double l1 = fabs(o.lam[0]), l5 = fabs(o.lam[4]);
      double sp = l1 > l5 ? l1 : l5;
      if (sp > Sx) Sx = sp;
      /* A- goes to the left cell, A+ to the right cell; (H, Hu, Hv, Z) */
      if (i - 1 >= 0) {
        double* a = acc + 4 * ((size_t)j * nx + (i - 1));
        a[0] += o.Am[0] / dx; a[1] += o.Am[1] / dx; a[2] += o.Am[2] / dx; a[3] += o.Am[3] / dx;
      }
      if (i < nx) {
        double* a = acc + 4 * ((size_t)j * nx + i);
        a[0] += o.Ap[0] / dx; a[1] += o.Ap[1] / dx; a[2] += o.Ap[2] / dx; a[3] += o.Ap[3] / dx;
      }
    }
  if (P->dim == 2) {
    /* y-interfaces j - 1/2, j = 0..ny; normal component = Hv */
    for (int j = 0; j <= ny; ++j)
      for (int i = 0; i < nx; ++i) {
        orc_cell L = orc_project_dir(P, X, i, j - 1, 1);
        orc_cell R = orc_project_dir(P, X, i, j, 1);
        double Lc[4], Rc[4];
        orc_conserved(X, i, j - 1, 1, Lc);
        orc_conserved(X, i, j, 1, Rc);
        int st = orc_solve(P, &L, &R, Lc, Rc, &o);
        if (st) return st;
        double l1 = fabs(o.lam[0]), l5 = fabs(o.lam[4]);
        double sp = l1 > l5 ? l1 : l5;
        if (sp > Sy) Sy = sp;
        /* back to (H, Hu, Hv, Z): comp 1 is Hv (normal), comp 2 is Hu */
        if (j - 1 >= 0) {
          double* a = acc + 4 * ((size_t)(j - 1) * nx + i);
          a[0] += o.Am[0] / dy; a[1] += o.Am[2] / dy; a[2] += o.Am[1] / dy; a[3] += o.Am[3] / dy;
        }
        if (j < ny) {
          double* a = acc + 4 * ((size_t)j * nx + i);
          a[0] += o.Ap[0] / dy; a[1] += o.Ap[2] / dy; a[2] += o.Ap[1] / dy; a[3] += o.Ap[3] / dy;
        }
      }
  }
  *Sx_out = Sx;
  *Sy_out = Sy;
  return ORC_OK;
}

/* The Godunov average of Sec. 3 in fluctuation form (forward Euler with the
 * net fluctuations acc of orc_ext_solve), then friction; the interior of X
 * is overwritten. */
static int orc_ext_update(const orc_params* P, orc_ext* X, double dt, const double* acc) {
  int nx = X->nx, ny = X->ny;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t c = (size_t)j * nx + i;
      size_t k = orc_xi(X, i, j);
      const double* a = acc + 4 * c;
      double Hn = X->H[k] - dt * a[0];
      double q1 = X->Hu[k] - dt * a[1];
      double q2 = (P->dim == 2) ? X->Hv[k] - dt * a[2] : 0.0;
      double Zn = X->Z[k] - dt * a[3];
      orc_friction(P, dt, Hn, &q1, &q2);
      int st = orc_check_cell(Hn, q1, q2, Zn);
      if (st) return st;
      X->H[k] = Hn;
      X->Hu[k] = q1;
      X->Hv[k] = q2;
      X->Z[k] = Zn;
    }
  return ORC_OK;
}

/* One step of the scheme on (h, hu, hv, z) in place.  dt > 0 fixed, or
 * dt <= 0 for the CFL step; the step used is returned in *dt_used. */
static int orc_step(const orc_params* P, orc_ext* X, double dt_fixed, double* h, double* hu, double* hv, double* z,
                    double* dt_used, double* work /* 4 * nx * ny accumulators */) {
  int nx = X->nx, ny = X->ny;
  orc_fill(P, X, h, hu, hv, z);
  int st = orc_ext_check(P, X);
  if (st) return st;
  double Sx, Sy;
  st = orc_ext_solve(P, X, work, &Sx, &Sy);
  if (st) return st;
  double dt = dt_fixed > 0.0 ? dt_fixed : orc_dt_of_speeds(P, Sx, Sy);
  if (!(dt > 0.0) || !isfinite(dt)) return ORC_ERR_DT;
  *dt_used = dt;
  st = orc_ext_update(P, X, dt, work);
  if (st) return st;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t c = (size_t)j * nx + i;
      size_t k = orc_xi(X, i, j);
      h[c] = X->H[k];
      hu[c] = X->Hu[k];
      if (P->dim == 2) hv[c] = X->Hv[k];
      z[c] = X->Z[k];
    }
  return ORC_OK;
}

static int orc_check_params(const orc_params* P) {
  if (!P) return ORC_ERR_ARG;
  if (P->dim != 1 && P->dim != 2) return ORC_ERR_ARG;
  if (P->nx < 1 || P->ny < 1 || (P->dim == 1 && P->ny != 1)) return ORC_ERR_ARG;
  if (!(P->lx > 0.0) || (P->dim == 2 && !(P->ly > 0.0)) || !(P->g > 0.0)) return ORC_ERR_ARG;
  if (!(P->kappa_a > 1.0) || !(P->beta_min > 0.0) || !(P->gamma_z >= 0.0) || !(P->newton_tol > 0.0) ||
      P->newton_maxit < 1)
    return ORC_ERR_ARG;
  if (P->bedload < ORC_GRASS || P->bedload > ORC_CAMENEN) return ORC_ERR_ARG;
  if (P->bedload == ORC_GRASS && (P->m_g < 1.0 || P->A_g < 0.0)) return ORC_ERR_ARG;
  if (P->bedload != ORC_GRASS && (P->friction == ORC_FRIC_NONE || !(P->s > 1.0) || !(P->d_s > 0.0)))
    return ORC_ERR_ARG;
  if (P->friction == ORC_FRIC_STRICKLER && !(P->K_st > 0.0)) return ORC_ERR_ARG;
  for (int s = 0; s < (P->dim == 2 ? 4 : 2); ++s) {
    if (P->bc[s] < 0 || P->bc[s] > ORC_BC_WALL) return ORC_ERR_ARG;
  }
  if ((P->bc[0] == ORC_BC_PERIODIC) != (P->bc[1] == ORC_BC_PERIODIC)) return ORC_ERR_ARG;
  if (P->dim == 2 && (P->bc[2] == ORC_BC_PERIODIC) != (P->bc[3] == ORC_BC_PERIODIC)) return ORC_ERR_ARG;
  return ORC_OK;
}

/* ---- exported entry points --------------------------------------------- */

/* One interface solve.  Lc, Rc: conserved (H, H un, H ut, Z) of the left and
 * right cells in the interface's normal orientation. */
int orc_riemann(const orc_params* P, const double* Lc, const double* Rc, orc_riemann_out* out) {
  if (!P || !Lc || !Rc || !out) return ORC_ERR_ARG;
  if (!(Lc[0] > 0.0) || !(Rc[0] > 0.0)) return ORC_ERR_NEG_DEPTH;
  orc_cell L = orc_project(P, Lc[0], Lc[1], Lc[2], Lc[3]);
  orc_cell R = orc_project(P, Rc[0], Rc[1], Rc[2], Rc[3]);
  return orc_solve(P, &L, &R, Lc, Rc, out);
}

/* Closure and equilibrium projection of one state, for tests:
 * out = (tau, un, ut, Pi, Omega, dOmega/dun, ca, cb). */
int orc_cell_project(const orc_params* P, const double* c, double* out) {
  if (!P || !c || !out) return ORC_ERR_ARG;
  orc_cell q = orc_project(P, c[0], c[1], c[2], c[3]);
  double Q, dQ;
  orc_closure(P, c[0], q.un, q.ut, &Q, &dQ);
  out[0] = q.tau; out[1] = q.un; out[2] = q.ut; out[3] = q.Pi;
  out[4] = q.Om; out[5] = dQ; out[6] = q.ca; out[7] = q.cb;
  return ORC_OK;
}

/* CFL time step of a state (reading R5). */
int orc_cfl(const orc_params* P, const double* h, const double* hu, const double* hv, const double* z,
            double* dt_out) {
  int st = orc_check_params(P);
  if (st) return st;
  orc_ext X;
  if (orc_ext_alloc(&X, P->nx, P->ny)) { orc_ext_free(&X); return ORC_ERR_ARG; }
  orc_fill(P, &X, h, hu, P->dim == 2 ? hv : NULL, z);
  double* acc = malloc(sizeof(double) * 4 * (size_t)P->nx * P->ny);
  if (!acc) { orc_ext_free(&X); return ORC_ERR_ARG; }
  double Sx, Sy;
  st = orc_ext_solve(P, &X, acc, &Sx, &Sy);
  if (!st) *dt_out = orc_dt_of_speeds(P, Sx, Sy);
  free(acc);
  orc_ext_free(&X);
  return st;
}

/* nsteps steps in place.  dts: NULL for CFL steps, else the fixed step of
 * each step.  t (in/out) accumulates time.  dts_out (nullable) receives the
 * step sizes used.  diag (nullable, 2 * nsteps) receives sum(h) dx dy and
 * sum(z) dx dy after each step, summed in row-major order.  Returns 0 or
 * the first error; *done receives the number of completed steps. */
int orc_run(const orc_params* P, int nsteps, const double* dts, double* h, double* hu, double* hv, double* z,
            double* t, double* dts_out, double* diag, int* done) {
  int st = orc_check_params(P);
  if (st) return st;
  if (nsteps < 0 || !h || !hu || !z || (P->dim == 2 && !hv)) return ORC_ERR_ARG;
  int nx = P->nx, ny = P->ny;
  orc_ext X;
  if (orc_ext_alloc(&X, nx, ny)) { orc_ext_free(&X); return ORC_ERR_ARG; }
  double* work = malloc(sizeof(double) * 4 * (size_t)nx * ny);
  if (!work) { orc_ext_free(&X); return ORC_ERR_ARG; }
  double dx = P->lx / nx;
  double dy = (P->dim == 2) ? P->ly / ny : 1.0;
  int n;
  st = ORC_OK;
  for (n = 0; n < nsteps; ++n) {
    double dt_used = 0.0;
    st = orc_step(P, &X, dts ? dts[n] : 0.0, h, hu, P->dim == 2 ? hv : NULL, z, &dt_used, work);
    if (st) break;
    if (t) *t += dt_used;
    if (dts_out) dts_out[n] = dt_used;
    if (diag) {
      double mh = 0.0, mz = 0.0;
      for (size_t c = 0; c < (size_t)nx * ny; ++c) { mh += h[c]; mz += z[c]; }
      diag[2 * n] = mh * dx * dy;
      diag[2 * n + 1] = mz * dx * dy;
    }
  }
  if (done) *done = n;
  free(work);
  orc_ext_free(&X);
  return st;
}

/* ---- the splitting scheme (the approach the paper contrasts with its own) ----
 *
 * The end of Sec. 2 describes the usual alternative to the coupled method: a
 * shallow-water step over the time step, after which the Exner equation
 * updates the bed.  The paper gives no discretisation of it; this file takes
 * (reading R13):
 *   1. the shallow-water step: the step above with the transport switched off
 *      (the Grass law with A_g = 0, so Omega = 0 and dQ/du = 0: the relaxation
 *      solver for shallow water over the bed), its CFL time step from those
 *      waves, friction as in the step; the bed is held at z^n;
 *   2. the Exner step with the transport law of P and the new flow:
 *        z_i <- z_i - dt/dx (F_{i+1/2} - F_{i-1/2}) - dt/dy (G_{j+1/2} - G_{j-1/2}),
 *      the bedload flux at an interface being Q_s of the cell upwind of it
 *      by the sign of the sum of the two cells' normal velocities (the mean
 *      of both cells' where the sum is 0, so that a wall, whose ghost
 *      mirrors the normal velocity, passes no sediment), ghost cells by the
 *      boundary rules. */

/* Bedload flux through the interface between cells (iL, jL) and (iR, jR) of
 * X in the x (ydir = 0) or y direction: Q_s of the upwind cell, the mean of
 * both where the normal velocities cancel (a wall: zero). */
static double orc_exner_flux(const orc_params* P, const orc_ext* X, int iL, int jL, int iR, int jR, int ydir) {
  double cL[4], cR[4];
  orc_conserved(X, iL, jL, ydir, cL);
  orc_conserved(X, iR, jR, ydir, cR);
  double unL = cL[1] / cL[0], unR = cR[1] / cR[0];
  double s = unL + unR, QL = 0.0, QR = 0.0, dQ;
  if (s >= 0.0) orc_closure(P, cL[0], unL, cL[2] / cL[0], &QL, &dQ);
  if (s <= 0.0) orc_closure(P, cR[0], unR, cR[2] / cR[0], &QR, &dQ);
  if (s > 0.0) return QL;
  if (s < 0.0) return QR;
  return 0.5 * (QL + QR);
}

static int orc_split_step(const orc_params* P, orc_ext* X, double dt_fixed, double* h, double* hu, double* hv,
                          double* z, double* dt_used, double* work, double* zn) {
  int nx = X->nx, ny = X->ny;
  size_t n = (size_t)nx * ny;
  orc_params Psw = *P;
  Psw.bedload = ORC_GRASS;
  Psw.A_g = 0.0;
  Psw.m_g = 3.0;
  memcpy(zn, z, sizeof(double) * n);
  int st = orc_step(&Psw, X, dt_fixed, h, hu, hv, z, dt_used, work);
  if (st) return st;
  memcpy(z, zn, sizeof(double) * n); /* the bed held fixed through the shallow-water step */
  orc_fill(P, X, h, hu, hv, z);
  double dt = *dt_used, dx = orc_dx(P), dy = orc_dy(P);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double fe = orc_exner_flux(P, X, i, j, i + 1, j, 0);
      double fw = orc_exner_flux(P, X, i - 1, j, i, j, 0);
      double d = dt / dx * (fe - fw);
      if (P->dim == 2) {
        double gn = orc_exner_flux(P, X, i, j, i, j + 1, 1);
        double gs = orc_exner_flux(P, X, i, j - 1, i, j, 1);
        d += dt / dy * (gn - gs);
      }
      zn[(size_t)j * nx + i] = z[(size_t)j * nx + i] - d;
    }
  for (size_t c = 0; c < n; ++c) {
    if (!isfinite(zn[c])) return ORC_ERR_NAN;
    z[c] = zn[c];
  }
  return ORC_OK;
}

/* nsteps steps of the splitting scheme in place (arguments as orc_run). */
int orc_split_run(const orc_params* P, int nsteps, const double* dts, double* h, double* hu, double* hv, double* z,
                  double* t, double* dts_out, double* diag, int* done) {
  int st = orc_check_params(P);
  if (st) return st;
  if (nsteps < 0 || !h || !hu || !z || (P->dim == 2 && !hv)) return ORC_ERR_ARG;
  int nx = P->nx, ny = P->ny;
  orc_ext X;
  if (orc_ext_alloc(&X, nx, ny)) { orc_ext_free(&X); return ORC_ERR_ARG; }
  double* work = malloc(sizeof(double) * 5 * (size_t)nx * ny);
  if (!work) { orc_ext_free(&X); return ORC_ERR_ARG; }
  double dx = orc_dx(P), dy = orc_dy(P);
  int k;
  st = ORC_OK;
  for (k = 0; k < nsteps; ++k) {
    double dt_used = 0.0;
    st = orc_split_step(P, &X, dts ? dts[k] : 0.0, h, hu, P->dim == 2 ? hv : NULL, z, &dt_used, work,
                        work + 4 * (size_t)nx * ny);
    if (st) break;
    if (t) *t += dt_used;
    if (dts_out) dts_out[k] = dt_used;
    if (diag) {
      double mh = 0.0, mz = 0.0;
      for (size_t c = 0; c < (size_t)nx * ny; ++c) { mh += h[c]; mz += z[c]; }
      diag[2 * k] = mh * dx * dy;
      diag[2 * k + 1] = mz * dx * dy;
    }
  }
  if (done) *done = k;
  free(work);
  orc_ext_free(&X);
  return st;
}

/* Byte sizes of the exported structs, so a caller can check its mirror. */
int orc_sizeof_params(void) { return (int)sizeof(orc_params); }
int orc_sizeof_riemann_out(void) { return (int)sizeof(orc_riemann_out); }

/* ---- blocks of a domain decomposition (Sec. 4) ----------------------------
 * A block is a padded array (nxl + 2) x (nyl + 2) of each field (index
 * (j + 1)(nxl + 2) + (i + 1)), cut from the grid of P (P->nx, P->ny are the
 * whole grid's sizes and fix dx, dy).  The caller fills the ghost ring:
 * halo cells from the neighbouring blocks, or the boundary rule on the
 * block's physical sides (orc_block_ghost).  The arithmetic is the one the
 * whole-grid stepper uses, so a decomposed run equals it bit for bit. */

static orc_ext orc_block_view(int nxl, int nyl, double* H, double* Hu, double* Hv, double* Z) {
  orc_ext X;
  X.nx = nxl; X.ny = nyl; X.ex = nxl + 2;
  X.H = H; X.Hu = Hu; X.Hv = Hv; X.Z = Z;
  return X;
}

/* Boundary rule of side (0 W, 1 E, 2 S, 3 N) into the block's ghosts from
 * the block's adjacent interior cells (non-periodic sides only). */
int orc_block_ghost(const orc_params* P, int nxl, int nyl, double* H, double* Hu, double* Hv, double* Z, int side) {
  if (!P || nxl < 1 || nyl < 1 || side < 0 || side > 3 || P->bc[side] == ORC_BC_PERIODIC) return ORC_ERR_ARG;
  orc_ext X = orc_block_view(nxl, nyl, H, Hu, Hv, Z);
  double in[4], out[4];
  if (side < 2) {
    for (int j = 0; j < nyl; ++j) {
      orc_ext_get(&X, side == 0 ? 0 : nxl - 1, j, in);
      orc_ghost(P, side, in, out);
      orc_ext_put(&X, side == 0 ? -1 : nxl, j, out);
    }
  } else {
    for (int i = 0; i < nxl; ++i) {
      orc_ext_get(&X, i, side == 2 ? 0 : nyl - 1, in);
      orc_ghost(P, side, in, out);
      orc_ext_put(&X, i, side == 2 ? -1 : nyl, out);
    }
  }
  return ORC_OK;
}

/* One solve per interface of the block (ghosts filled by the caller): the
 * net fluctuation of each interior cell into work (4 nxl nyl doubles, owned
 * by the caller, read by orc_block_update) and the extreme wave speeds
 * (S[0] x, S[1] y) of the block's solves. */
int orc_block_solve(const orc_params* P, int nxl, int nyl, double* H, double* Hu, double* Hv, double* Z,
                    double* work, double* S) {
  if (!P || !S || !work || nxl < 1 || nyl < 1) return ORC_ERR_ARG;
  orc_ext X = orc_block_view(nxl, nyl, H, Hu, Hv, Z);
  int st = orc_ext_check(P, &X);
  if (st) return st;
  return orc_ext_solve(P, &X, work, &S[0], &S[1]);
}

/* CFL step of the whole grid from its extreme speeds. */
int orc_block_dt(const orc_params* P, double Sx, double Sy, double* dt) {
  if (!P || !dt) return ORC_ERR_ARG;
  *dt = orc_dt_of_speeds(P, Sx, Sy);
  return (*dt > 0.0 && isfinite(*dt)) ? ORC_OK : ORC_ERR_DT;
}

/* One step of size dt on the block's interior from the net fluctuations
 * orc_block_solve left in work for the same state. */
int orc_block_update(const orc_params* P, int nxl, int nyl, double* H, double* Hu, double* Hv, double* Z,
                     const double* work, double dt) {
  if (!P || !work || nxl < 1 || nyl < 1 || !(dt > 0.0)) return ORC_ERR_ARG;
  orc_ext X = orc_block_view(nxl, nyl, H, Hu, Hv, Z);
  return orc_ext_update(P, &X, dt, work);
}
