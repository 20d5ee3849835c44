// Test driver: the reverse-mode transposed-Jacobian product of one
// interface's fluctuations (interface_vjp) against the forward-mode
// dual-number passes (jac_pass), on inputs read from stdin.
// Input per line: HL HnL HtL ZL HR HnR HtR ZR A m Am0..Am3 Ap0..Ap3
// (18 numbers).  Output per line: ok, then the 10 forward-mode values, then
// the 10 reverse-mode values, then the number of negative wave speeds,
// whether the bed-step bound set a, the Newton updates, the doublings of a,
// the halved Newton steps and the spread of the specific volumes
// max / min over tauL, tau1..tau4, tauR.
#include <cstdio>
#include <cstring>
#include <vector>

#include "../paper_1307_0491_gb300/csrc/sve_adjoint_jac.cuh"

using namespace sve;

__global__ void vjp_pairs(DevParams P, const double* in, double* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* x = in + 18 * i;
  double* o = out + 27 * i;
  const double u[8] = {x[0], x[1], x[2], x[3], x[4], x[5], x[6], x[7]};
  const double A = x[8], m = x[9];
  const double Amb[4] = {x[10], x[11], x[12], x[13]}, Apb[4] = {x[14], x[15], x[16], x[17]};
  const Cell<double> L = project_grass<double>(P, u[0], u[1], u[2], u[3], A, m);
  const Cell<double> R = project_grass<double>(P, u[4], u[5], u[6], u[7], A, m);
  double a, b;
  const bool raised = celerities(P, L, R, a, b);
  const double tol = 16.0 * 2.220446049250313e-16 > P.newton_tol ? 16.0 * 2.220446049250313e-16 : P.newton_tol;
  NewtonConst<double> c;
  NewtonEval<double> e;
  double p = 0.0;
  int its = 0, halv = 0, retries = 0;
  bool ok = false;
  for (;; ++retries) {  // the solve of the step, with its doublings of a
    p = newton_setup(P, L, R, a, b, c);
    newton_eval(p, c, L, R, e);
    ok = newton_loop(c, L, R, p, e, P.newton_maxit, tol, its, halv) && newton_positive(e);
    if (ok || retries == kARetries) break;
    a = 2.0 * a;
  }
  o[0] = ok ? 1.0 : 0.0;
  if (!ok) return;
  const double Fp = newton_deriv(c, e);
  double fwd[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  jac_pass<0>(P, u, A, m, p, Fp, Amb, Apb, 1.0, fwd, retries);
  jac_pass<1>(P, u, A, m, p, Fp, Amb, Apb, 1.0, fwd, retries);
  double ub[8] = {0, 0, 0, 0, 0, 0, 0, 0}, Ab = 0.0, mb = 0.0, Kb = 0.0;
  if (!interface_vjp(P, u, A, m, Amb, Apb, ub, Ab, mb, Kb)) o[0] = 0.0;
  for (int k = 0; k < 10; ++k) o[1 + k] = fwd[k];
  for (int k = 0; k < 8; ++k) o[11 + k] = ub[k];
  o[19] = Ab;
  o[20] = mb;
  // diagnostics: the fan state and the celerity branch
  NewtonEval<double> ee;
  newton_eval(p, c, L, R, ee);
  newton_fill(c, L, ee);  // u1, u4, Z* at the root
  const double lam1 = L.un - a * L.tau, lam5 = R.un + a * R.tau, us = ee.u1 + b * (ee.tau2 - ee.tau1);
  o[21] = (double)((lam1 < 0) + (ee.lam2 < 0) + (us < 0) + (ee.lam4 < 0) + (lam5 < 0));
  o[22] = raised ? 1.0 : 0.0;
  o[23] = (double)its;
  o[24] = (double)retries;
  o[25] = (double)halv;
  const double tmn = fmin(fmin(fmin(ee.tau1, ee.tau2), fmin(ee.tau3, ee.tau4)), fmin(L.tau, R.tau));
  const double tmx = fmax(fmax(fmax(ee.tau1, ee.tau2), fmax(ee.tau3, ee.tau4)), fmax(L.tau, R.tau));
  o[26] = tmx / tmn;
}

int main() {
  std::vector<double> in;
  double v;
  while (std::scanf("%lf", &v) == 1) in.push_back(v);
  const int n = (int)(in.size() / 18);
  if (n == 0 || in.size() % 18) return 1;
  DevParams P;
  std::memset(&P, 0, sizeof(P));
  P.dim = 2;
  P.g = 9.81;
  P.inv_2g = 1.0 / (2.0 * 9.81);
  P.kappa_a = 1.1;
  P.beta_min = 0.01;
  P.gamma_z = 2.0;
  P.two_g = 2.0 * 9.81;
  P.two_g_gamma = 2.0 * 9.81 * 2.0;
  P.newton_tol = 1e-9;
  P.newton_maxit = 30;
  P.bedload = 0;
  double *din = nullptr, *dout = nullptr;
  if (cudaMalloc(&din, sizeof(double) * in.size()) != cudaSuccess) return 2;
  if (cudaMalloc(&dout, sizeof(double) * 27 * (size_t)n) != cudaSuccess) return 2;
  cudaMemcpy(din, in.data(), sizeof(double) * in.size(), cudaMemcpyHostToDevice);
  cudaMemset(dout, 0, sizeof(double) * 27 * (size_t)n);
  vjp_pairs<<<(n + 127) / 128, 128>>>(P, din, dout, n);
  std::vector<double> out(27 * (size_t)n);
  if (cudaMemcpy(out.data(), dout, sizeof(double) * out.size(), cudaMemcpyDeviceToHost) != cudaSuccess) return 3;
  for (int i = 0; i < n; ++i) {
    for (int k = 0; k < 27; ++k) std::printf(k ? " %.17g" : "%.17g", out[27 * i + k]);
    std::printf("\n");
  }
  cudaFree(din);
  cudaFree(dout);
  return 0;
}
