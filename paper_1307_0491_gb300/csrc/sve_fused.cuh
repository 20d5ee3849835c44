// sve_fused.cuh -- the FP32-state 2D step as a shared-memory stencil.
//
// In FP32 the two-launch layout of sve_device.cuh (projection and
// fluctuations through global memory) is bound by its load/store stream, not
// by arithmetic; this form keeps the projection and the fluctuations on
// chip.  Per step:
//   solve_kernel   a tile of TX x TY cells plus its one-cell halo is staged
//                  and projected in shared memory; every x- and y-interface
//                  of the tile is solved once (the Riemann solver of
//                  sve_device.cuh), its fluctuations kept in shared memory,
//                  and each cell's net fluctuation dF = (A+ of the left and
//                  lower interface + A- of the right and upper one) / dx, dy
//                  is written out (16 B per cell; it does not depend on the
//                  time step).  The extreme wave speeds come from the solves
//                  themselves; the last block to finish turns their running
//                  maximum into the time step, as interface_kernel does;
//   apply_kernel   U <- U - dt dF per cell, semi-implicit friction, checks,
//                  the ghosts, per-block mass partials; in place, bound by
//                  its 48 B per cell of HBM traffic.
// Both kernels are launched with as many blocks as fit on the GPU at once and
// walk their tiles / cells with a grid stride, so that the per-block partials
// stay few.  Interfaces on tile edges are solved by both neighbouring tiles
// (8 % more solves at 32 x 8), the price of keeping fluctuations off HBM.
#pragma once
#include "sve_device.cuh"

namespace sve {

// 32 x 8 cells per tile; 288 threads solve the tile's 8 x 33 + 9 x 32 = 552
// interfaces in two rounds, the first 256 of them update its cells.
constexpr int kFTX = 32, kFTY = 8, kFCells = kFTX * kFTY, kFThreads = 288;
constexpr int kFSX = kFTX + 2, kFSY = kFTY + 2;  // staged tile with halo
constexpr int kFNX = kFTY * (kFTX + 1), kFNY = (kFTY + 1) * kFTX;

// Conserved state of one buffer (padded (ny + 2) x (nx + 2)).
template <typename T>
struct StateBuf {
  T *h, *hu, *hv, *z;
};

// Projected cell in shared memory (x-normal orientation; the y frame swaps).
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
  c.cbx = tsqrt(Hu * Hu + g * H * H * dQx);
  c.cby = P.dim == 2 ? tsqrt(Hv * Hv + g * H * H * dQy) : T(0);
}

template <typename T>
__device__ __forceinline__ Cell<T> frame_cell(const SCell<T>& s, bool ydir) {
  Cell<T> c;
  c.H = s.H; c.Z = s.Z; c.tau = s.tau; c.Pi = s.Pi; c.ca = s.ca;
  if (!ydir) { c.Hn = s.Hu; c.Ht = s.Hv; c.un = s.u; c.ut = s.v; c.Om = s.omx; c.cb = s.cbx; }
  else { c.Hn = s.Hv; c.Ht = s.Hu; c.un = s.v; c.ut = s.u; c.Om = s.omy; c.cb = s.cby; }
  return c;
}

// Stage and project the tile (bx, by) with its halo: smem cell (li, lj) is
// the grid cell (i0 - 1 + li, j0 - 1 + lj); cells outside the padded grid and
// the four halo corners are not used.
template <typename T>
__device__ __forceinline__ void stage_tile(const DevParams& P, const StateBuf<T>& B, int i0, int j0,
                                           SCell<T> (*sc)[kFSX]) {
  for (int k = threadIdx.x; k < kFSX * kFSY; k += kFThreads) {
    const int lj = k / kFSX, li = k - lj * kFSX;
    const int i = i0 - 1 + li, j = j0 - 1 + lj;
    const bool corner = (li == 0 || li == kFSX - 1) && (lj == 0 || lj == kFSY - 1);
    const bool inside = i >= -1 && i <= P.nx && j >= (P.dim == 2 ? -1 : 0) && j <= (P.dim == 2 ? P.ny : 0);
    if (corner || !inside) continue;
    const long long e = ext_index(P, i, j);
    project_into(P, B.h[e], B.hu[e], P.dim == 2 ? B.hv[e] : T(0), B.z[e], sc[lj][li]);
  }
  __syncthreads();
}

// Interface k of a tile (x-interfaces first): its smem cells (li, lj) on the
// right / top and the grid indices (i, j) of that cell; false if the
// interface is outside the grid.
__device__ __forceinline__ bool tile_interface(const DevParams& P, int i0, int j0, int k, bool& ydir, int& li,
                                               int& lj) {
  ydir = k >= kFNX;
  if (!ydir) { lj = 1 + k / (kFTX + 1); li = 1 + k % (kFTX + 1); }
  else { const int q = k - kFNX; lj = 1 + q / kFTX; li = 1 + q % kFTX; }
  const int i = i0 - 1 + li, j = j0 - 1 + lj;
  // interface (i - 1/2, j) for x, (i, j - 1/2) for y
  return !ydir ? (i <= P.nx && j < P.ny) : (i < P.nx && j <= P.ny);
}

// Max over the block of non-negative floats held as their bit patterns
// (integer order = float order for them; a NaN wins, as in the two-launch form).
__device__ __forceinline__ unsigned block_max_u32(unsigned v, unsigned* sh) {
  v = __reduce_max_sync(0xffffffffu, v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  unsigned r = 0u;
#pragma unroll
  for (int w = 0; w < kFThreads / 32; ++w) r = max(r, sh[w]);
  __syncthreads();
  return r;
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
  if ((!perx && i == 0) || (perx && i == P.nx - 1)) { ghost_state(P, 0, s, gs); put(-1, j); }
  if ((!perx && i == P.nx - 1) || (perx && i == 0)) { ghost_state(P, 1, s, gs); put(P.nx, j); }
  if (P.dim == 2) {
    const bool pery = P.bc[2] == GHOST_PERIODIC;
    if ((!pery && j == 0) || (pery && j == P.ny - 1)) { ghost_state(P, 2, s, gs); put(i, -1); }
    if ((!pery && j == P.ny - 1) || (pery && j == 0)) { ghost_state(P, 3, s, gs); put(i, P.ny); }
  }
}


// Net fluctuation planes of the solve (unpadded nx x ny, component-major).
template <typename T>
struct NetFluct {
  T *h, *hu, *hv, *z;
};

template <typename T>
__global__ void __launch_bounds__(kFThreads, 3) solve_kernel(DevParams P, StateBuf<T> B, NetFluct<T> D,
                                                             DevScalars* sc, const double* fixed_dts,
                                                             double* dtlog, int fixed, int ntiles, int tiles_x) {
  static_assert(sizeof(T) == 4, "the fused step is the FP32 form");
  __shared__ SCell<T> cells[kFSY][kFSX];
  // fluctuations, component-major so that neighbouring threads hit
  // neighbouring banks: [c] = A- (c < 4) and A+ (c >= 4) of (H, Hn, Ht, Z)
  __shared__ T fx[8][kFTY][kFTX + 1];
  __shared__ T fy[8][kFTY + 1][kFTX];
  __shared__ unsigned int s_sx, s_sy, s_its, s_warps, s_halv, s_raised, s_retry;
  if (threadIdx.x == 0) { s_sx = 0u; s_sy = 0u; s_its = 0u; s_warps = 0u; s_halv = 0u; s_raised = 0u; s_retry = 0u; }
  __syncthreads();
  const T idx = par<T>(P.inv_dx, (float)P.inv_dx), idy = par<T>(P.inv_dy, (float)P.inv_dy);
  const int tx = threadIdx.x % kFTX, ty = threadIdx.x / kFTX;  // cell of this thread (ty < TY)
  int fail = 0, iters = 0;
  unsigned int nraised = 0u, nretry = 0u, nhalv = 0u;
  unsigned int mx = 0u, my = 0u;  // speed maxima (bit patterns of non-negative floats)
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int i0 = (t % tiles_x) * kFTX, j0 = (t / tiles_x) * kFTY;
    stage_tile(P, B, i0, j0, cells);  // ends with a barrier
    for (int k = threadIdx.x; k < kFNX + kFNY; k += kFThreads) {
      bool ydir;
      int li, lj;
      if (!tile_interface(P, i0, j0, k, ydir, li, lj)) continue;
      const Cell<T> L = frame_cell(!ydir ? cells[lj][li - 1] : cells[lj - 1][li], ydir);
      const Cell<T> R = frame_cell(cells[lj][li], ydir);
      T Am[4], Ap[4], smax;
      int its = 0, branch = 0;
      if (!riemann_solve(P, L, R, Am, Ap, smax, its, branch)) fail = 1;
      iters += its;
      nraised += branch_raised(branch);
      nretry += branch_retries(branch);
      nhalv += branch_halvings(branch);
      const unsigned int sb = __float_as_uint(smax);
      if (!ydir) {
        mx = max(mx, sb);
#pragma unroll
        for (int c = 0; c < 4; ++c) { fx[c][lj - 1][li - 1] = Am[c]; fx[4 + c][lj - 1][li - 1] = Ap[c]; }
      } else {
        my = max(my, sb);
#pragma unroll
        for (int c = 0; c < 4; ++c) { fy[c][lj - 1][li - 1] = Am[c]; fy[4 + c][lj - 1][li - 1] = Ap[c]; }
      }
    }
    __syncthreads();
    const int i = i0 + tx, j = j0 + ty;
    if (ty < kFTY && i < P.nx && j < P.ny) {
      // A+ of the interface on the left / bottom plus A- of the one on the
      // right / top (the y fluctuations are in the y frame: Hn = Hv)
      const long long o = (long long)j * P.nx + i;
      D.h[o] = (fx[4][ty][tx] + fx[0][ty][tx + 1]) * idx + (fy[4][ty][tx] + fy[0][ty + 1][tx]) * idy;
      D.hu[o] = (fx[5][ty][tx] + fx[1][ty][tx + 1]) * idx + (fy[6][ty][tx] + fy[2][ty + 1][tx]) * idy;
      D.hv[o] = (fx[6][ty][tx] + fx[2][ty][tx + 1]) * idx + (fy[5][ty][tx] + fy[1][ty + 1][tx]) * idy;
      D.z[o] = (fx[7][ty][tx] + fx[3][ty][tx + 1]) * idx + (fy[7][ty][tx] + fy[3][ty + 1][tx]) * idy;
    }
    __syncthreads();  // the next tile overwrites cells and fluctuations
  }
  if (fail) atomicOr(&sc->status, ST_RIEMANN);
  // tallies: warp shuffles, shared-memory atomics, the block's last warp
  // folds them into the step's running maxima (as interface_kernel does)
  mx = __reduce_max_sync(0xffffffffu, mx);
  my = __reduce_max_sync(0xffffffffu, my);
  iters = __reduce_add_sync(0xffffffffu, iters);
  nraised = __reduce_add_sync(0xffffffffu, nraised);
  nhalv = __reduce_add_sync(0xffffffffu, nhalv);
  nretry = __reduce_add_sync(0xffffffffu, nretry);
  if ((threadIdx.x & 31) != 0) return;
  atomicMax(&s_sx, mx);
  atomicMax(&s_sy, my);
  atomicAdd(&s_its, (unsigned int)iters);
  if (nraised | nretry | nhalv) { atomicAdd(&s_raised, nraised); atomicAdd(&s_retry, nretry); atomicAdd(&s_halv, nhalv); }
  __threadfence_block();
  if (atomicAdd(&s_warps, 1u) != kFThreads / 32 - 1) return;
  __threadfence_block();
  const double bx = (double)__uint_as_float(atomicMax(&s_sx, 0u));
  const double by = (double)__uint_as_float(atomicMax(&s_sy, 0u));
  atomicAdd(&sc->newton_iters, (unsigned long long)atomicAdd(&s_its, 0u));
  const unsigned br = atomicAdd(&s_raised, 0u), bt = atomicAdd(&s_retry, 0u), bh = atomicAdd(&s_halv, 0u);
  if (bt) atomicAdd(&sc->retries, (unsigned long long)bt);
  if (br) atomicAdd(&sc->raised, (unsigned long long)br);
  if (bh) atomicAdd(&sc->halvings, (unsigned long long)bh);
  atomicMax(&sc->smax_bits[0], (unsigned long long)__double_as_longlong(bx));
  atomicMax(&sc->smax_bits[1], (unsigned long long)__double_as_longlong(by));
  __threadfence();
  if (atomicAdd(&sc->done_iface, 1u) != gridDim.x - 1) return;
  __threadfence();
  const double sx = __longlong_as_double((long long)atomicExch(&sc->smax_bits[0], 0ull));
  const double sy = __longlong_as_double((long long)atomicExch(&sc->smax_bits[1], 0ull));
  const int cs = sc->call_step;
  double dt;
  if (fixed) dt = fixed_dts[cs];
  else if (P.dim == 1) dt = P.cfl * P.dx / sx;
  else dt = P.cfl / (sx / P.dx + sy / P.dy);
  if (!(dt > 0.0) || !isfinite(dt)) { atomicOr(&sc->status, ST_DT); dt = 0.0; }
  sc->dt = dt;
  sc->Sx = sx;
  sc->Sy = sy;
  dtlog[cs] = dt;
  sc->done_iface = 0u;
}

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

constexpr int kAThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kAThreads) apply_kernel(DevParams P, StateBuf<T> B, NetFluct<T> D,
                                                          DevScalars* sc, double* mpart, Mirror<T> out) {
  static_assert(sizeof(T) == 4, "the fused step is the FP32 form");
  __shared__ double s_m[2][kAThreads];
  __shared__ unsigned int s_warps;
  if (threadIdx.x == 0) s_warps = 0u;
  __syncthreads();
  const T dt = T(sc->dt);
  int st = 0;
  FSum sh_h, sh_z;
  // rows by a grid stride in y, columns by a grid stride in x
  for (int j = blockIdx.y; j < P.ny; j += gridDim.y) {
    for (int i = blockIdx.x * kAThreads + threadIdx.x; i < P.nx; i += gridDim.x * kAThreads) {
      const long long e = ext_index(P, i, j), k = (long long)j * P.nx + i;
      T s[4] = {B.h[e] - dt * D.h[k], B.hu[e] - dt * D.hu[k], B.hv[e] - dt * D.hv[k], B.z[e] - dt * D.z[k]};
      if (P.friction != 0) {
        const T tau = tdiv(T(1), s[0]);
        const T qn = tsqrt(s[1] * s[1] + s[2] * s[2]);
        T C = par<T>(P.fric_c, P.f.fric_c) * (tau * tau);
        if (P.friction == 2) C = C * rcbrt64(s[0]);
        const T den = T(1) + dt * C * qn;
        s[1] = tdiv(s[1], den);
        s[2] = tdiv(s[2], den);
      }
      if (!(finite_bits(s[0]) && finite_bits(s[1]) && finite_bits(s[2]) && finite_bits(s[3]))) st |= ST_NAN;
      else if (!positive(s[0])) st |= ST_NEG_DEPTH;
      B.h[e] = s[0]; B.hu[e] = s[1]; B.hv[e] = s[2]; B.z[e] = s[3];
      if (out.h) { out.h[k] = s[0]; out.hu[k] = s[1]; out.hv[k] = s[2]; out.z[k] = s[3]; }
      write_ghost_state(P, B, i, j, s);
      sh_h.add(s[0]);
      sh_z.add(s[3]);
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
