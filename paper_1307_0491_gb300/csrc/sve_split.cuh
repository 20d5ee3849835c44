// sve_split.cuh -- the splitting scheme (FP64): the approach the paper's
// Sec. 2 contrasts with its coupled method -- a shallow-water step over the
// time step, after which the Exner equation updates the bed.
//
// The paper gives no discretisation of it; the library takes:
//   1. the shallow-water step: the coupled step of sve_device.cuh with the
//      transport switched off (the Grass law with A_g = 0: Omega = 0,
//      dQ/du = 0, so the relaxation solver is one for shallow water over the
//      bed), its CFL time step from those waves, friction as in the step,
//      the bed held at z^n (the step's own bed update is discarded: its
//      b-waves move a non-flat bed a little even without transport);
//   2. exner_kernel: the Exner update with the configured transport law and
//      the new flow, z_i <- z_i - dt/dx (F_{i+1/2} - F_{i-1/2})
//      - dt/dy (G_{j+1/2} - G_{j-1/2}), the bedload flux at an interface
//      being Q_s of the cell upwind of it by the sign of the sum of the two
//      cells' normal velocities (the mean of both where the sum is 0, so a
//      wall, whose ghost mirrors the normal velocity, passes no sediment);
//      ghost cells by the boundary rules.
#pragma once
#include "sve_device.cuh"

namespace sve {

// Bedload flux through the interface between padded cells eL and eR, in the
// x (ydir false) or y frame, from the new flow in S.
__device__ __forceinline__ double exner_flux(const DevParams& P, const DevState<double>& S, long long eL,
                                             long long eR, bool ydir) {
  const double* hn = ydir ? S.hv : S.hu;
  const double* ht = ydir ? S.hu : S.hv;
  const double HL = S.h[eL], HR = S.h[eR];
  const double unL = hn[eL] / HL, unR = hn[eR] / HR;
  const double s = unL + unR;
  double QL = 0.0, QR = 0.0, dQ;
  if (s >= 0.0) closure(P, HL, unL, P.dim == 2 ? ht[eL] / HL : 0.0, QL, dQ);
  if (s <= 0.0) closure(P, HR, unR, P.dim == 2 ? ht[eR] / HR : 0.0, QR, dQ);
  if (s > 0.0) return QL;
  if (s < 0.0) return QR;
  return 0.5 * (QL + QR);
}

// One interior cell k per thread, the launch shape of cell_kernel<double, NT>
// (so that the block's bed-mass partial replaces the one the cell kernel
// wrote, summed in the same order): the new bed from the held bed z0
// (padded), the time step in sc->dt; the ghosts' bed by the boundary rules
// (every rule copies the bed).
template <int NT>
__global__ void __launch_bounds__(NT) exner_kernel(DevParams P, DevState<double> S, const double* z0,
                                                   DevScalars* sc, double* mpart) {
  __shared__ double s_m[NT];
  __shared__ unsigned int s_warps;
  if (threadIdx.x == 0) s_warps = 0u;
  __syncthreads();
  const long long k = (long long)blockIdx.x * NT + threadIdx.x;
  const long long ncell = (long long)P.nx * P.ny;
  double mz = 0.0;
  if (k < ncell) {
    const int j = (int)(k / P.nx), i = (int)(k - (long long)j * P.nx);
    const long long e = ext_index(P, i, j);
    const double dt = sc->dt;
    const double fe = exner_flux(P, S, e, e + 1, false), fw = exner_flux(P, S, e - 1, e, false);
    double d = dt * P.inv_dx * (fe - fw);
    if (P.dim == 2) {
      const double gn = exner_flux(P, S, e, e + P.ex, true), gs = exner_flux(P, S, e - P.ex, e, true);
      d += dt * P.inv_dy * (gn - gs);
    }
    const double z = z0[e] - d;
    if (!finite_bits(z)) atomicOr(&sc->status, ST_NAN);
    S.z[e] = z;
    const bool perx = P.bc[0] == GHOST_PERIODIC;
    if ((!perx && i == 0) || (perx && i == P.nx - 1)) S.z[ext_index(P, -1, j)] = z;
    if ((!perx && i == P.nx - 1) || (perx && i == 0)) S.z[ext_index(P, P.nx, j)] = z;
    if (P.dim == 2) {
      const bool pery = P.bc[2] == GHOST_PERIODIC;
      if ((!pery && j == 0) || (pery && j == P.ny - 1)) S.z[ext_index(P, i, -1)] = z;
      if ((!pery && j == P.ny - 1) || (pery && j == 0)) S.z[ext_index(P, i, P.ny)] = z;
    }
    mz = z;
  }
  // the block's bed-mass partial (as cell_kernel sums it)
  s_m[threadIdx.x] = mz;
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
  double b = 0.0;
#pragma unroll
  for (int q = 0; q < NT / 32; ++q) b += s_m[lane + 32 * q];
  b = warp_sum(b);
  if (lane == 0) mpart[2 * blockIdx.x + 1] = b;
}

}  // namespace sve
