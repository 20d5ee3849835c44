// sve_fused.cuh -- the FP32-state 2D step as a fused stencil: shared
// pieces and the apply pass.
//
// In FP32 the two-launch layout of sve_device.cuh (projection and
// fluctuations through global memory) is bound by its load/store stream, not
// by arithmetic; the fused form keeps the projection and the fluctuations on
// chip.  Per step:
//   solve pass     (march_kernel, sve_march.cuh) the state is projected and
//                  every interface solved on chip (the Riemann solver of
//                  sve_device.cuh); each cell's net fluctuation dF = (A+ of
//                  the left and lower interface + A- of the right and upper
//                  one) / dx, dy is written out (16 B per cell; it does not
//                  depend on the time step); the extreme wave speeds come
//                  from the solves and the last block turns their running
//                  maximum into the time step, as interface_kernel does;
//   apply_kernel   U <- U - dt dF per cell, semi-implicit friction, checks,
//                  the ghosts, per-block mass partials; in place (or from a
//                  second state buffer), bound by its 48 B per cell of HBM
//                  traffic (a grid stride over rows and columns with as many
//                  blocks as fit at once, so that the per-block partials
//                  stay few).
// Within one call of several steps, the update of step n is instead applied
// by the solve pass of step n + 1 as it reads the state (march_kernel's
// carried form, sve_march.cuh), and the apply pass runs once, after the last
// solve pass.
#pragma once
#include "sve_device.cuh"

namespace sve {

// Conserved state of one buffer (padded (ny + 2) x (nx + 2)).
template <typename T>
struct StateBuf {
  T *h, *hu, *hv, *z;
};

// Projected cell (x-normal orientation; the y frame swaps).
template <typename T>
struct SCell {
  T H, Hu, Hv, Z, tau, u, v, Pi, omx, omy, ca, cbx, cby;
};

template <typename T>
__device__ __forceinline__ void project_into(const DevParams& P, T H, T Hu, T Hv, T Z, SCell<T>& c) {
  c.H = H; c.Hu = Hu; c.Hv = Hv; c.Z = Z;
  c.tau = tdiv(T(1), H);
  c.u = Hu * c.tau;
  c.v = Hv * c.tau;
  const T g = par<T>(P.g, P.f.g);
  c.Pi = T(0.5) * g * H * H;
  T Qx, dQx, Qy = T(0), dQy = T(0);
  if (P.dim == 2) closure2(P, H, c.u, c.v, Qx, dQx, Qy, dQy);
  else closure(P, H, c.u, c.v, Qx, dQx);
  c.omx = Qx;
  c.omy = Qy;
  c.ca = H * tsqrt(g * H);
  c.cbx = tsqrt(tfma(Hu, Hu, g * H * H * dQx));
  c.cby = P.dim == 2 ? tsqrt(tfma(Hv, Hv, g * H * H * dQy)) : T(0);
}

template <typename T>
__device__ __forceinline__ Cell<T> frame_cell(const SCell<T>& s, bool ydir) {
  Cell<T> c;
  c.H = s.H; c.Z = s.Z; c.tau = s.tau; c.Pi = s.Pi; c.ca = s.ca;
  if (!ydir) { c.Hn = s.Hu; c.Ht = s.Hv; c.un = s.u; c.ut = s.v; c.Om = s.omx; c.cb = s.cbx; }
  else { c.Hn = s.Hv; c.Ht = s.Hu; c.un = s.v; c.ut = s.u; c.Om = s.omy; c.cb = s.cby; }
  return c;
}

// Ghost cells of the new state fed by cell (i, j) (conserved fields only).
template <typename T>
__device__ __forceinline__ void write_ghost_state(const DevParams& P, const StateBuf<T>& B, int i, int j,
                                                  const T s[4]) {
  T gs[4];
  auto put = [&](int gi, int gj) {
    const long long e = ext_index(P, gi, gj);
    B.h[e] = gs[0]; B.hu[e] = gs[1]; B.hv[e] = gs[2]; B.z[e] = gs[3];
  };
  const bool perx = P.bc[0] == GHOST_PERIODIC;
  if (((!perx && i == 0) || (perx && i == P.nx - 1)) && P.bc[0] != GHOST_EXTERNAL) { ghost_state(P, 0, s, gs); put(-1, j); }
  if (((!perx && i == P.nx - 1) || (perx && i == 0)) && P.bc[1] != GHOST_EXTERNAL) { ghost_state(P, 1, s, gs); put(P.nx, j); }
  if (P.dim == 2) {
    const bool pery = P.bc[2] == GHOST_PERIODIC;
    if (((!pery && j == 0) || (pery && j == P.ny - 1)) && P.bc[2] != GHOST_EXTERNAL) { ghost_state(P, 2, s, gs); put(i, -1); }
    if (((!pery && j == P.ny - 1) || (pery && j == 0)) && P.bc[3] != GHOST_EXTERNAL) { ghost_state(P, 3, s, gs); put(i, P.ny); }
  }
}


// Net fluctuation planes of the solve (unpadded nx x ny, component-major).
template <typename T>
struct NetFluct {
  T *h, *hu, *hv, *z;
};

// Compensated (Neumaier) FP32 running sum: s + c carries the sum of the
// values to O(n eps^2), so the per-thread mass partials need no FP64 adds
// (an FP64 add per cell and field would load the FP64 pipe, ~1/64 of FP32).
struct FSum {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float x) {
    const float t = s + x;
    c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// Plain running sum for the FP64 state.
struct DSum {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};
template <typename T> struct MassSum { using type = DSum; };
template <> struct MassSum<float> { using type = FSum; };

constexpr int kAThreads = 256;

// The new state of one cell from its state u and net fluctuation d: U <-
// U - dt dF, then the semi-implicit friction (every product written as the
// FMA it is, so that every kernel that applies an update -- the apply pass,
// the solve pass applying the previous step's -- gives the same bits).
template <typename T>
__device__ __forceinline__ void apply_state(const DevParams& P, T dt, const T u[4], const T d[4], T s[4]) {
#pragma unroll
  for (int c = 0; c < 4; ++c) s[c] = tfma(-dt, d[c], u[c]);
  if (P.friction != 0) {
    const T tau = tdiv(T(1), s[0]);
    const T qn = tsqrt(tfma(s[1], s[1], s[2] * s[2]));
    T C = par<T>(P.fric_c, P.f.fric_c) * (tau * tau);
    if (P.friction == 2) C = C * rcbrt64(s[0]);
    const T den = tfma(dt * C, qn, T(1));
    s[1] = tdiv(s[1], den);
    s[2] = tdiv(s[2], den);
  }
}

// Status bits of a new state: non-finite, or a non-positive depth.
template <typename T>
__device__ __forceinline__ int state_check(const T s[4]) {
  if (!(finite_bits(s[0]) && finite_bits(s[1]) && finite_bits(s[2]) && finite_bits(s[3]))) return ST_NAN;
  return positive(s[0]) ? 0 : ST_NEG_DEPTH;
}

// The update of one interior cell (i, j) from its net fluctuation: the state
// of src plus the update into dst (src == dst: in place), checks, the ghosts
// it feeds (in dst), the optional mirror; returns status bits, (mh, mz) = the
// new (h, z).
template <typename T>
__device__ __forceinline__ int apply_cell(const DevParams& P, const StateBuf<T>& src, const StateBuf<T>& dst,
                                          const NetFluct<T>& D, T dt, int i, int j, const Mirror<T>& out, T& mh,
                                          T& mz) {
  const long long e = ext_index(P, i, j), k = (long long)j * P.nx + i;
  const T u[4] = {src.h[e], src.hu[e], src.hv[e], src.z[e]};
  const T d[4] = {D.h[k], D.hu[k], D.hv[k], D.z[k]};
  T s[4];
  apply_state(P, dt, u, d, s);
  const int st = state_check(s);
  dst.h[e] = s[0]; dst.hu[e] = s[1]; dst.hv[e] = s[2]; dst.z[e] = s[3];
  if (out.h) { out.h[k] = s[0]; out.hu[k] = s[1]; out.hv[k] = s[2]; out.z[k] = s[3]; }
  write_ghost_state(P, dst, i, j, s);
  mh = s[0];
  mz = s[3];
  return st;
}

// src: the state the update applies to; B: where the new state goes (the
// same buffer: in place).
template <typename T>
__global__ void __launch_bounds__(kAThreads) apply_kernel(DevParams P, StateBuf<T> src, StateBuf<T> B,
                                                          NetFluct<T> D, DevScalars* sc, double* mpart,
                                                          Mirror<T> out) {
  __shared__ double s_m[2][kAThreads];
  __shared__ unsigned int s_warps;
  if (threadIdx.x == 0) s_warps = 0u;
  __syncthreads();
  const T dt = T(sc->dt);
  int st = 0;
  typename MassSum<T>::type sh_h, sh_z;
  // rows by a grid stride in y, columns by a grid stride in x
  for (int j = blockIdx.y; j < P.ny; j += gridDim.y) {
    for (int i = blockIdx.x * kAThreads + threadIdx.x; i < P.nx; i += gridDim.x * kAThreads) {
      T mh, mz;
      st |= apply_cell(P, src, B, D, dt, i, j, out, mh, mz);
      sh_h.add(mh);
      sh_z.add(mz);
    }
  }
  if (st) atomicOr(&sc->status, st);
  // the block's mass partial in a fixed order by its last warp (as in cell_kernel)
  s_m[0][threadIdx.x] = sh_h.value();
  s_m[1][threadIdx.x] = sh_z.value();
  __syncwarp();
  unsigned int w = 0u;
  if ((threadIdx.x & 31) == 0) {
    __threadfence_block();
    w = atomicAdd(&s_warps, 1u);
  }
  w = __shfl_sync(0xffffffffu, w, 0);
  if (w != kAThreads / 32 - 1) return;
  __threadfence_block();
  const int lane = threadIdx.x & 31;
  double a = 0.0, b = 0.0;
#pragma unroll
  for (int q = 0; q < kAThreads / 32; ++q) { a += s_m[0][lane + 32 * q]; b += s_m[1][lane + 32 * q]; }
  a = warp_sum(a);
  b = warp_sum(b);
  if (lane != 0) return;
  const unsigned int bid = blockIdx.y * gridDim.x + blockIdx.x, nb = gridDim.x * gridDim.y;
  mpart[2 * bid] = a;
  mpart[2 * bid + 1] = b;
  __threadfence();
  if (atomicAdd(&sc->done_cell, 1u) != nb - 1) return;
  // the step is complete (mass sums: from the partials on read-out)
  sc->mass_parts = nb;
  sc->t += sc->dt;
  sc->call_step += 1;
  sc->steps += 1;
  sc->done_cell = 0u;
}

}  // namespace sve
