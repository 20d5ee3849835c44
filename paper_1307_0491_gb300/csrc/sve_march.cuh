// sve_march.cuh -- the solve pass of the FP32-state 2D step as register
// stencils marching along column strips.
//
// One warp owns a strip of 30 interior columns plus one halo column on each
// side (lane l <-> column x0 - 1 + l) and walks a run of rows j0..j1-1.  Per
// row it projects its cell of the next row (Pi = g h^2 / 2, Omega = q_b: the
// lambda -> 0 projection of Sec. 3), solves the y-interface between the
// current and the next row at its column and the x-interface on its left
// (the left neighbour's projected cell comes by warp shuffles), takes the
// right interface's A- from its right neighbour by a shuffle, and writes the
// cell's net fluctuation dF = (A+ left + A- right) / dx + (A+ below + A- above)
// / dy -- the below term carried in registers from the previous row.  No
// shared memory and no block barrier: every warp is independent, the state
// is read once per strip (the two halo columns are read by both neighbouring
// strips, 1/15 more reads), and each interface is solved once except the
// strip edges' x-interfaces (1/30 more) and one row of y-interfaces per run
// of rows.  The extreme wave speeds come from the solves and the last block
// turns them into the time step, as in the other solve passes.
#pragma once
#include "sve_fused.cuh"

namespace sve {

constexpr int kMCols = 30;    // interior columns per strip (32 lanes: 30 + two halo columns)
constexpr int kMWarps = 4;    // warps per block
constexpr int kMThreads = 32 * kMWarps;

// Runs of rows per strip: as many rows per warp as give every SM its 20
// resident warps (five 4-warp blocks), at least 4 rows (the one extra row of
// y-solves per run costs 1/rows) and at most 32 (on the 8192 x 4096
// antidune runs of 32 rows measured 2.3 % faster than 64 and 1.6 % faster
// than 16; warps drawing their runs from a ticket counter instead of one run
// per warp made no difference).
struct MarchShape {
  int strips, rows, chunks;
  long long tasks;
  unsigned blocks;
};

inline MarchShape march_shape(const DevParams& P, int nsm) {
  MarchShape M;
  M.strips = (P.nx + kMCols - 1) / kMCols;
  const long long want = 20LL * nsm;  // warps in flight
  long long rows = ((long long)M.strips * P.ny + want - 1) / want;
  rows = rows < 4 ? 4 : (rows > 32 ? 32 : rows);
  M.rows = (int)rows;
  M.chunks = (P.ny + M.rows - 1) / M.rows;
  M.tasks = (long long)M.strips * M.chunks;
  M.blocks = (unsigned)((M.tasks + kMWarps - 1) / kMWarps);
  return M;
}

// Running maximum of non-negative wave speeds held as bit patterns (integer
// order = IEEE order for them): 32-bit in FP32, 64-bit in FP64; the warp
// maximum as the double value's bit pattern.
template <typename T> struct SpeedMax;
template <> struct SpeedMax<float> {
  unsigned v = 0u;
  __device__ __forceinline__ void add(float s) { v = max(v, __float_as_uint(s)); }
  __device__ __forceinline__ unsigned long long warp_bits() const {
    return (unsigned long long)__double_as_longlong((double)__uint_as_float(__reduce_max_sync(0xffffffffu, v)));
  }
};
template <> struct SpeedMax<double> {
  unsigned long long v = 0ull;
  __device__ __forceinline__ void add(double s) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(s);
    v = b > v ? b : v;
  }
  __device__ __forceinline__ unsigned long long warp_bits() const {
    unsigned long long b = v;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ob = __shfl_xor_sync(0xffffffffu, b, o);
      b = ob > b ? ob : b;
    }
    return b;
  }
};

// The carried update: within a call of several steps the solve pass of step
// n + 1 reads U^n and the net fluctuations of step n and applies the update
// itself (apply_state, bit for bit the apply pass's), so that the state makes
// one trip through memory per step instead of two.
template <typename T>
struct Carry {
  StateBuf<T> dst;  // where the owning lanes store U^{n+1} (interior cells; not the ghosts)
  NetFluct<T> D;    // the net fluctuations of step n
  T dt;             // the time step of step n
};

// U^{n+1} of padded cell (c, j) from U^n in B and the carried update:
// interior cells by apply_state, ghost cells by their side's ghost rule from
// the cell they copy (as write_ghost_state fills them: the first or last
// interior cell, the far one across a periodic side), corners (never solved
// with) a unit state.  No external sides.
template <typename T>
__device__ __forceinline__ void carried_state(const DevParams& P, const StateBuf<T>& B, const Carry<T>& K, int c,
                                              int j, T s[4]) {
  const bool xin = c >= 0 && c < P.nx, yin = j >= 0 && j < P.ny;
  int side = -1, i0 = c, j0 = j;
  if (!xin && !yin) {
    s[0] = T(1); s[1] = T(0); s[2] = T(0); s[3] = T(0);
    return;
  }
  if (!xin) {
    const bool per = P.bc[0] == GHOST_PERIODIC;
    side = c < 0 ? 0 : 1;
    i0 = (c < 0) != per ? 0 : P.nx - 1;
  } else if (!yin) {
    const bool per = P.bc[2] == GHOST_PERIODIC;
    side = j < 0 ? 2 : 3;
    j0 = (j < 0) != per ? 0 : P.ny - 1;
  }
  const long long e = ext_index(P, i0, j0), k = (long long)j0 * P.nx + i0;
  const T u[4] = {B.h[e], B.hu[e], B.hv[e], B.z[e]};
  const T d[4] = {K.D.h[k], K.D.hu[k], K.D.hv[k], K.D.z[k]};
  if (side < 0) {
    apply_state(P, K.dt, u, d, s);
  } else {
    T a[4];
    apply_state(P, K.dt, u, d, a);
    // (a runtime side: the rule's component indices make this a small
    // local-memory array; dispatching on constant sides measured 2 % slower)
    ghost_state(P, side, a, s);
  }
}

// The x-frame cell of the lane below (lane - 1) by shuffles.
template <typename T>
__device__ __forceinline__ Cell<T> left_cell(const SCell<T>& s) {
  Cell<T> c;
  const unsigned m = 0xffffffffu;
  c.H = __shfl_up_sync(m, s.H, 1);
  c.Hn = __shfl_up_sync(m, s.Hu, 1);
  c.Ht = __shfl_up_sync(m, s.Hv, 1);
  c.Z = __shfl_up_sync(m, s.Z, 1);
  c.tau = __shfl_up_sync(m, s.tau, 1);
  c.un = __shfl_up_sync(m, s.u, 1);
  c.ut = __shfl_up_sync(m, s.v, 1);
  c.Pi = __shfl_up_sync(m, s.Pi, 1);
  c.Om = __shfl_up_sync(m, s.omx, 1);
  c.ca = __shfl_up_sync(m, s.ca, 1);
  c.cb = __shfl_up_sync(m, s.cbx, 1);
  return c;
}

// Tallies of one thread's solves: failures, Newton updates, safeguards,
// extreme speeds of the x- and y-solves.
template <typename T>
struct MarchTally {
  int fail = 0, iters = 0, status = 0;
  unsigned int nraised = 0u, nretry = 0u, nhalv = 0u;
  SpeedMax<T> mx, my;
};

// One task: the strip `strip` (columns strip * 30 .. + 29 with a halo column
// each side) over the run of rows `chunk` (rows chunk * rows ..), by the
// calling warp (every lane must call it).  carry: B holds U^n and the
// carried update K gives the state the step solves with (the task's own
// cells stored into K.dst and checked).  One code path for both (a runtime
// switch and a single projection site), so that the solves of a carried
// step are the same instructions as those of a plain one, bit for bit.
template <typename T>
__device__ __forceinline__ void march_task(const DevParams& P, const StateBuf<T>& B, const NetFluct<T>& D,
                                           int strip, int chunk, int rows, MarchTally<T>& t, bool carry = false,
                                           const Carry<T>& K = Carry<T>{}) {
  const int lane = threadIdx.x & 31;
  const int c = strip * kMCols - 1 + lane;          // this lane's column
  const bool col_in = c <= P.nx;                    // inside the padded grid
  const bool interior = lane >= 1 && lane <= kMCols && c < P.nx;  // a cell this strip updates
  const bool xface = lane >= 1 && col_in;           // the x-interface c - 1/2 exists
  const int j0 = chunk * rows, j1 = min(j0 + rows, P.ny);
  const T idx = par<T>(P.inv_dx, (float)P.inv_dx), idy = par<T>(P.inv_dy, (float)P.inv_dy);
  SCell<T> cur, nxt;
  T apb[4] = {T(0), T(0), T(0), T(0)};  // A+ of the y-interface below (j - 1/2), y frame
  // the projected cell of this lane's column at row jj (with the carried
  // update: the updated state, stored by the lane that owns the cell)
  auto project_row = [&](int jj, SCell<T>& out) {
    T a[4] = {T(1), T(0), T(0), T(0)};  // outside the padded grid: a unit state (never solved with)
    if (col_in) {
      if (carry) {
        carried_state(P, B, K, c, jj, a);
      } else {
        const long long e = ext_index(P, c, jj);
        a[0] = B.h[e]; a[1] = B.hu[e]; a[2] = B.hv[e]; a[3] = B.z[e];
      }
    }
    project_into(P, a[0], a[1], a[2], a[3], out);
    if (carry && interior && jj >= j0 && jj < j1) {
      const long long e = ext_index(P, c, jj);
      K.dst.h[e] = a[0]; K.dst.hu[e] = a[1]; K.dst.hv[e] = a[2]; K.dst.z[e] = a[3];
      t.status |= state_check(a);
    }
  };
  project_row(j0 - 1, cur);
  // j = j0 - 1 only solves the y-interface j0 - 1/2 (its A+ enters row j0)
  for (int j = j0 - 1; j < j1; ++j) {
    project_row(j + 1, nxt);
    const bool row = j >= j0;  // row j is updated by this task (warp-uniform)
    // the y-interface j + 1/2 at this column
    T amu[4] = {T(0), T(0), T(0), T(0)}, apu[4] = {T(0), T(0), T(0), T(0)};
    if (interior) {
      T s = T(0);
      int its = 0, br = 0;
      if (!riemann_solve(P, frame_cell(cur, true), frame_cell(nxt, true), amu, apu, s, its, br)) t.fail = 1;
      t.my.add(s);
      t.iters += its;
      t.nraised += branch_raised(br);
      t.nretry += branch_retries(br);
      t.nhalv += branch_halvings(br);
    }
    if (row) {
      // the x-interface c - 1/2 of row j; its A- goes to the lane below
      const Cell<T> L = left_cell(cur);
      T amx[4] = {T(0), T(0), T(0), T(0)}, apx[4] = {T(0), T(0), T(0), T(0)};
      if (xface) {
        T s = T(0);
        int its = 0, br = 0;
        if (!riemann_solve(P, L, frame_cell(cur, false), amx, apx, s, its, br)) t.fail = 1;
        t.mx.add(s);
        t.iters += its;
        t.nraised += branch_raised(br);
        t.nretry += branch_retries(br);
        t.nhalv += branch_halvings(br);
      }
      T amr[4];  // A- of the x-interface c + 1/2 (the right neighbour's)
#pragma unroll
      for (int k = 0; k < 4; ++k) amr[k] = __shfl_down_sync(0xffffffffu, amx[k], 1);
      if (interior) {
        // the y fluctuations are in the y frame: (H, Hv, Hu, Z)
        const long long o = (long long)j * P.nx + c;
        D.h[o] = (apx[0] + amr[0]) * idx + (apb[0] + amu[0]) * idy;
        D.hu[o] = (apx[1] + amr[1]) * idx + (apb[2] + amu[2]) * idy;
        D.hv[o] = (apx[2] + amr[2]) * idx + (apb[1] + amu[1]) * idy;
        D.z[o] = (apx[3] + amr[3]) * idx + (apb[3] + amu[3]) * idy;
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) apb[k] = apu[k];
    cur = nxt;
  }
}

// The block's tallies (every thread calls it): over the warp by reductions,
// over the block by shared-memory atomics, the block's last warp folds them
// into the run's scalars and returns true for that warp's lane 0 (false
// elsewhere).
template <typename T>
__device__ __forceinline__ bool march_fold(const MarchTally<T>& t, DevScalars* sc, unsigned long long* s_sx,
                                           unsigned long long* s_sy, unsigned int* s_cnt) {
  if (t.fail) atomicOr(&sc->status, ST_RIEMANN);
  if (t.status) atomicOr(&sc->status, t.status);
  const unsigned long long wx = t.mx.warp_bits(), wy = t.my.warp_bits();
  const unsigned iters = __reduce_add_sync(0xffffffffu, (unsigned)t.iters);
  const unsigned nraised = __reduce_add_sync(0xffffffffu, t.nraised);
  const unsigned nhalv = __reduce_add_sync(0xffffffffu, t.nhalv);
  const unsigned nretry = __reduce_add_sync(0xffffffffu, t.nretry);
  if ((threadIdx.x & 31) != 0) return false;
  // s_cnt: Newton updates, raised, doublings, halvings, warps done
  atomicMax(s_sx, wx);
  atomicMax(s_sy, wy);
  atomicAdd(&s_cnt[0], iters);
  if (nraised | nretry | nhalv) { atomicAdd(&s_cnt[1], nraised); atomicAdd(&s_cnt[2], nretry); atomicAdd(&s_cnt[3], nhalv); }
  __threadfence_block();
  if (atomicAdd(&s_cnt[4], 1u) != blockDim.x / 32 - 1) return false;
  __threadfence_block();
  atomicAdd(&sc->newton_iters, (unsigned long long)atomicAdd(&s_cnt[0], 0u));
  const unsigned br = atomicAdd(&s_cnt[1], 0u), bt = atomicAdd(&s_cnt[2], 0u), bh = atomicAdd(&s_cnt[3], 0u);
  if (br) atomicAdd(&sc->raised, (unsigned long long)br);
  if (bt) atomicAdd(&sc->retries, (unsigned long long)bt);
  if (bh) atomicAdd(&sc->halvings, (unsigned long long)bh);
  atomicMax(&sc->smax_bits[0], atomicMax(s_sx, 0ull));
  atomicMax(&sc->smax_bits[1], atomicMax(s_sy, 0ull));
  return true;
}

// Five blocks per SM (<= 102 registers a thread, no spills): 20 warps per SM
// measured 5 % faster than the unconstrained 123 registers (16 warps) and
// than six blocks (<= 85 registers) on the 8192 x 4096 antidune.
// carry: the carried form (B holds U^n; carry_dst, carry_D: where U^{n+1}
// goes and the net fluctuations of step n, whose time the finalizer accounts
// for before it takes step n + 1's time step).
template <typename T>
__global__ void __launch_bounds__(kMThreads, 5) march_kernel(DevParams P, StateBuf<T> B, NetFluct<T> D,
                                                          DevScalars* sc, const double* fixed_dts, double* dtlog,
                                                          int fixed, int strips, int rows, long long ntasks,
                                                          int carry = 0, StateBuf<T> carry_dst = StateBuf<T>{},
                                                          NetFluct<T> carry_D = NetFluct<T>{}) {
  __shared__ unsigned long long s_sx, s_sy;
  __shared__ unsigned int s_cnt[5];
  if (threadIdx.x == 0) { s_sx = 0ull; s_sy = 0ull; for (int k = 0; k < 5; ++k) s_cnt[k] = 0u; }
  __syncthreads();
  const long long task = (long long)blockIdx.x * kMWarps + (threadIdx.x >> 5);
  MarchTally<T> t;
  const Carry<T> K{carry_dst, carry_D, carry ? T(sc->dt) : T(0)};
  if (task < ntasks) march_task(P, B, D, (int)(task % strips), (int)(task / strips), rows, t, carry != 0, K);
  if (!march_fold(t, sc, &s_sx, &s_sy, s_cnt)) return;
  __threadfence();
  if (atomicAdd(&sc->done_iface, 1u) != gridDim.x - 1) return;
  __threadfence();
  const double sx = __longlong_as_double((long long)atomicExch(&sc->smax_bits[0], 0ull));
  const double sy = __longlong_as_double((long long)atomicExch(&sc->smax_bits[1], 0ull));
  if (carry) {
    // the carried step is complete (its mass sums: from the final apply pass)
    sc->t += sc->dt;
    sc->call_step += 1;
    sc->steps += 1;
  }
  const int cs = sc->call_step;
  double dt;
  if (fixed == DT_FIXED) dt = fixed_dts[cs];
  else if (fixed == DT_SPEEDS_ONLY) dt = 0.0;  // set by the caller from all blocks' speeds
  else dt = P.cfl / (sx / P.dx + sy / P.dy);
  if (fixed != DT_SPEEDS_ONLY && (!(dt > 0.0) || !isfinite(dt))) { atomicOr(&sc->status, ST_DT); dt = 0.0; }
  sc->dt = dt;
  sc->Sx = sx;
  sc->Sy = sy;
  dtlog[cs] = dt;
  sc->done_iface = 0u;
}

}  // namespace sve
