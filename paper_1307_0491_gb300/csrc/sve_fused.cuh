// sve_fused.cuh -- the FP32-state 2D step as a shared-memory stencil.
//
// In FP32 the two-launch layout of sve_device.cuh (projection and
// fluctuations through global memory) is bound by its load/store stream, not
// by arithmetic; this form keeps everything but the state on chip.  Per step:
//   speed_kernel   a tile of TX x TY cells plus its one-cell halo is staged
//                  and projected in shared memory; the extreme wave speeds of
//                  the tile's interfaces give per-block maxima; the last block
//                  to finish turns them into the time step (as the interface
//                  kernel of the two-launch form does);
//   fused_kernel   the same tile is staged and projected again, every x- and
//                  y-interface of the tile is solved once (the Riemann solver
//                  of sve_device.cuh), the fluctuations stay in shared memory,
//                  and each cell is updated, friction applied and the new
//                  state (and its ghosts) written to the other buffer of a
//                  double-buffered state; per-block mass partials.
// Both kernels are launched with as many blocks as fit on the GPU at once and
// walk the tiles with a grid stride, so that the per-block partials (and the
// serial work of the last block, which reduces them) stay small.
// Interfaces on tile edges are solved by both neighbouring tiles (8 % more
// solves at 32 x 8), the price of keeping fluctuations out of global memory.
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

template <typename T>
__global__ void __launch_bounds__(kFThreads, 7) speed_kernel(DevParams P, StateBuf<T> B, DevScalars* sc,
                                                          double* spart, const double* fixed_dts, double* dtlog,
                                                          int fixed, int ntiles, int tiles_x) {
  static_assert(sizeof(T) == 4, "the fused step is the FP32 form");
  __shared__ SCell<T> cells[kFSY][kFSX];
  __shared__ unsigned sh[kFThreads / 32];
  __shared__ bool last;
  unsigned mx = 0u, my = 0u;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int i0 = (t % tiles_x) * kFTX, j0 = (t / tiles_x) * kFTY;
    stage_tile(P, B, i0, j0, cells);
    for (int k = threadIdx.x; k < kFNX + kFNY; k += kFThreads) {
      bool ydir;
      int li, lj;
      if (!tile_interface(P, i0, j0, k, ydir, li, lj)) continue;
      const Cell<T> L = frame_cell(!ydir ? cells[lj][li - 1] : cells[lj - 1][li], ydir);
      const Cell<T> R = frame_cell(cells[lj][li], ydir);
      T a, b;
      celerities(P, L, R, a, b);
      const unsigned s = __float_as_uint(nnmax(absbits(L.un - a * L.tau), absbits(R.un + a * R.tau)));
      if (!ydir) mx = max(mx, s);
      else my = max(my, s);
    }
    __syncthreads();  // the next tile overwrites the staged cells
  }
  mx = block_max_u32(mx, sh);
  my = block_max_u32(my, sh);
  unsigned* up = reinterpret_cast<unsigned*>(spart);
  if (threadIdx.x == 0) {
    up[2 * blockIdx.x] = mx;
    up[2 * blockIdx.x + 1] = my;
    __threadfence();
    last = atomicAdd(&sc->done_iface, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  mx = 0u;
  my = 0u;
#pragma unroll 4
  for (unsigned q = threadIdx.x; q < gridDim.x; q += kFThreads) {
    mx = max(mx, __ldcg(up + 2 * q));
    my = max(my, __ldcg(up + 2 * q + 1));
  }
  mx = block_max_u32(mx, sh);
  my = block_max_u32(my, sh);
  if (threadIdx.x == 0) {
    const double sx = (double)__uint_as_float(mx), sy = (double)__uint_as_float(my);
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

template <typename T>
__global__ void __launch_bounds__(kFThreads, 3) fused_kernel(DevParams P, StateBuf<T> B, StateBuf<T> N,
                                                          DevScalars* sc, double* mpart, int ntiles, int tiles_x) {
  static_assert(sizeof(T) == 4, "the fused step is the FP32 form");
  __shared__ SCell<T> cells[kFSY][kFSX];
  // fluctuations, component-major so that neighbouring threads hit
  // neighbouring banks: [c] = A- (c < 4) and A+ (c >= 4) of (H, Hn, Ht, Z)
  __shared__ T fx[8][kFTY][kFTX + 1];
  __shared__ T fy[8][kFTY + 1][kFTX];
  __shared__ double sh[2 * (kFThreads / 32)];
  __shared__ bool last;
  const double dt = sc->dt;
  const T dtx = T(dt * P.inv_dx), dty = T(dt * P.inv_dy), dtT = T(dt);
  const int tx = threadIdx.x % kFTX, ty = threadIdx.x / kFTX;  // cell of this thread (ty < TY)
  int fail = 0, iters = 0, st = 0;
  FSum sh_h, sh_z;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int i0 = (t % tiles_x) * kFTX, j0 = (t / tiles_x) * kFTY;
    stage_tile(P, B, i0, j0, cells);
    for (int k = threadIdx.x; k < kFNX + kFNY; k += kFThreads) {
      bool ydir;
      int li, lj;
      if (!tile_interface(P, i0, j0, k, ydir, li, lj)) continue;
      const Cell<T> L = frame_cell(!ydir ? cells[lj][li - 1] : cells[lj - 1][li], ydir);
      const Cell<T> R = frame_cell(cells[lj][li], ydir);
      T Am[4], Ap[4], s;
      int its = 0;
      if (!riemann_solve(P, L, R, Am, Ap, s, its)) fail = 1;
      iters += its;
      if (!ydir) {
#pragma unroll
        for (int c = 0; c < 4; ++c) { fx[c][lj - 1][li - 1] = Am[c]; fx[4 + c][lj - 1][li - 1] = Ap[c]; }
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) { fy[c][lj - 1][li - 1] = Am[c]; fy[4 + c][lj - 1][li - 1] = Ap[c]; }
      }
    }
    __syncthreads();
    const int i = i0 + tx, j = j0 + ty;
    if (ty < kFTY && i < P.nx && j < P.ny) {
      const SCell<T>& c0 = cells[ty + 1][tx + 1];
      // A+ of the interface on the left / bottom plus A- of the one on the
      // right / top (the y fluctuations are in the y frame: Hn = Hv)
      T s[4] = {c0.H, c0.Hu, c0.Hv, c0.Z};
      const T ax0 = fx[4][ty][tx] + fx[0][ty][tx + 1], ax1 = fx[5][ty][tx] + fx[1][ty][tx + 1];
      const T ax2 = fx[6][ty][tx] + fx[2][ty][tx + 1], ax3 = fx[7][ty][tx] + fx[3][ty][tx + 1];
      const T ay0 = fy[4][ty][tx] + fy[0][ty + 1][tx], ay1 = fy[5][ty][tx] + fy[1][ty + 1][tx];
      const T ay2 = fy[6][ty][tx] + fy[2][ty + 1][tx], ay3 = fy[7][ty][tx] + fy[3][ty + 1][tx];
      s[0] = s[0] - (dtx * ax0 + dty * ay0);
      s[1] = s[1] - (dtx * ax1 + dty * ay2);
      s[2] = s[2] - (dtx * ax2 + dty * ay1);
      s[3] = s[3] - (dtx * ax3 + dty * ay3);
      if (P.friction != 0) {
        const T tau = tdiv(T(1), s[0]);
        const T qn = tsqrt(s[1] * s[1] + s[2] * s[2]);
        T C = par<T>(P.fric_c, P.f.fric_c) * (tau * tau);
        if (P.friction == 2) C = C * rcbrt64(s[0]);
        const T den = T(1) + dtT * C * qn;
        s[1] = tdiv(s[1], den);
        s[2] = tdiv(s[2], den);
      }
      if (!(finite_bits(s[0]) && finite_bits(s[1]) && finite_bits(s[2]) && finite_bits(s[3]))) st |= ST_NAN;
      else if (!positive(s[0])) st |= ST_NEG_DEPTH;
      const long long e = ext_index(P, i, j);
      N.h[e] = s[0]; N.hu[e] = s[1]; N.hv[e] = s[2]; N.z[e] = s[3];
      write_ghost_state(P, N, i, j, s);
      sh_h.add(s[0]);
      sh_z.add(s[3]);
    }
    __syncthreads();  // the next tile overwrites cells and fluctuations
  }
  if (fail) atomicOr(&sc->status, ST_RIEMANN);
  if (st) atomicOr(&sc->status, st);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) iters += __shfl_xor_sync(0xffffffffu, iters, o);
  if ((threadIdx.x & 31) == 0 && iters) atomicAdd(&sc->newton_iters, (unsigned long long)iters);
  double mh = sh_h.value(), mz = sh_z.value();
  block_sum2<kFThreads>(mh, mz, sh);
  if (threadIdx.x == 0) {
    mpart[2 * blockIdx.x] = mh;
    mpart[2 * blockIdx.x + 1] = mz;
    __threadfence();
    last = atomicAdd(&sc->done_cell, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  // the step is complete (mass sums: from the partials on read-out)
  sc->mass_parts = gridDim.x;
  sc->t += sc->dt;
  sc->call_step += 1;
  sc->steps += 1;
  sc->done_cell = 0u;
}

}  // namespace sve
