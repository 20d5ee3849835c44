// sve_persist.cuh -- the step of small grids as one persistent cooperative
// launch for many steps.
//
// On a grid of a few thousand cells a step's two kernel launches are the
// same order of time as its work.  Here one cooperative launch of one-warp
// blocks (all co-resident, spread over the SMs so that the FP64 work is
// too) runs a whole batch of steps; inside a step the two phases of the
// two-kernel form are separated by grid-wide barriers:
//   A  every interface solved once (Sec. 3: the relaxation Riemann problem
//      and its fluctuations), the extreme wave speeds max-reduced;
//   -- barrier --  every block takes the same CFL dt from the maxima;
//   B  every cell updated (Godunov average, friction, projection, ghosts);
//   -- barrier --
// The per-interface and per-cell arithmetic is that of interface_kernel and
// cell_kernel (the same device functions), so the states and time steps
// equal the two-kernel path's up to round-off (each kernel is compiled on
// its own, and the compiler may contract a multiply-add differently); the
// mass-sum partials are added in another order.  Every wait of the barrier is bounded: past the limit a
// block latches ST_SYNC and leaves, every other block then runs out of its
// own waits, and the host reads the status (the context stays usable).
// Measured on GB300 it is no faster than the two kernels from CUDA graphs
// (1D dune, 1000 cells: 40.2 k against 40.3 k steps/s; a barrier costs
// 1.9 us, and a step is bound by one warp's chain of ~300 FP64 instructions
// at the SM sub-partition's FP64 rate, which the graph launches overlap), so
// it is opt-in.
#pragma once

#include "sve_device.cuh"

namespace sve {

constexpr int ST_SYNC = 16;              // status bit: a grid-wide wait ran out
constexpr int kPersistThreads = 32;      // one warp per block
constexpr long long kBarrierPolls = 1LL << 22;  // bounded wait (~0.5 s of polling)

// Device scratch of the persistent step (zeroed before each launch).
struct PersistScratch {
  unsigned int count;                  // blocks arrived at the current barrier
  unsigned int gen;                    // barrier generation (released when it changes)
  unsigned long long smax[2][2];       // [step parity][x, y] running maxima of the speeds (bit patterns)
};

// Grid-wide barrier over the launch's blocks (all co-resident: cooperative
// launch), `expected` arrivals releasing it.  Thread 0 of each block arrives
// and waits; the wait polls at most `polls` times.  Returns false (in every
// thread of the block) if the wait ran out.
__device__ __forceinline__ bool grid_barrier(PersistScratch* ps, unsigned int expected, unsigned int& gen,
                                             long long polls) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned int g = gen;
    __threadfence();
    if (atomicAdd(&ps->count, 1u) == expected - 1u) {
      atomicExch(&ps->count, 0u);
      __threadfence();
      atomicExch(&ps->gen, g + 1u);
    } else {
      long long n = 0;
      while (*(volatile unsigned int*)&ps->gen == g) {
        if (++n > polls) {
          ok = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    gen = g + 1u;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// nsteps steps of a grid whose interfaces and cells the launch's blocks
// cover by a grid stride.  fixed: dt from fixed_dts[call_step] instead of
// the CFL condition.  expected: the barrier's arrivals (gridDim.x; larger
// only to exercise the bounded wait).
template <typename T>
__global__ void __launch_bounds__(kPersistThreads, 1) persistent_kernel(DevParams P, DevState<T> S, DevScalars* sc,
                                                                     PersistScratch* ps, const double* fixed_dts,
                                                                     double* dtlog, int fixed, int nsteps,
                                                                     double* mpart, unsigned int expected,
                                                                     long long polls) {
  unsigned int gen = 0u;
  const int cs0 = sc->call_step;
  const long long nf = P.nfx + P.nfy;
  const long long ncell = (long long)P.nx * P.ny;
  const long long stride = (long long)gridDim.x * kPersistThreads;
  const long long t0 = (long long)blockIdx.x * kPersistThreads + threadIdx.x;
  for (int st = 0; st < nsteps; ++st) {
    const int par = st & 1;
    // A: interfaces
    long long bx = 0, by = 0;
    int iters = 0, nraised = 0, nretry = 0, nhalv = 0;
    int bad = 0;
    for (long long idx = t0; idx < nf; idx += stride) {
      const bool ydir = idx >= P.nfx;
      const long long k = ydir ? idx - P.nfx : idx;
      double smax = 0.0;
      int it = 0, branch = 0;
      if (!interface_item(P, S, ydir, k, smax, it, branch)) bad = ST_RIEMANN;
      iters += it;
      nraised += (int)branch_raised(branch);
      nretry += (int)branch_retries(branch);
      nhalv += (int)branch_halvings(branch);
      const long long b = __double_as_longlong(smax);  // speeds are >= 0: integer order = IEEE order
      if (ydir) by = b > by ? b : by;
      else bx = b > bx ? b : bx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const long long ox = __shfl_xor_sync(0xffffffffu, bx, o), oy = __shfl_xor_sync(0xffffffffu, by, o);
      bx = ox > bx ? ox : bx;
      by = oy > by ? oy : by;
      iters += __shfl_xor_sync(0xffffffffu, iters, o);
      bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    nraised = (int)__reduce_add_sync(0xffffffffu, (unsigned)nraised);
    nhalv = (int)__reduce_add_sync(0xffffffffu, (unsigned)nhalv);
    nretry = (int)__reduce_add_sync(0xffffffffu, (unsigned)nretry);
    if (threadIdx.x == 0) {
      if (bad) atomicOr(&sc->status, bad);
      atomicAdd(&sc->newton_iters, (unsigned long long)iters);
      if (nraised) atomicAdd(&sc->raised, (unsigned long long)nraised);
      if (nhalv) atomicAdd(&sc->halvings, (unsigned long long)nhalv);
      if (nretry) atomicAdd(&sc->retries, (unsigned long long)nretry);
      atomicMax(&ps->smax[par][0], (unsigned long long)bx);
      atomicMax(&ps->smax[par][1], (unsigned long long)by);
    }
    if (!grid_barrier(ps, expected, gen, polls)) {
      if (threadIdx.x == 0) atomicOr(&sc->status, ST_SYNC);
      return;
    }
    // every block: the step's dt from the maxima (read from L2)
    const double sx = __longlong_as_double((long long)atomicOr(&ps->smax[par][0], 0ull));
    const double sy = __longlong_as_double((long long)atomicOr(&ps->smax[par][1], 0ull));
    const int cs = cs0 + st;
    double dt;
    if (fixed) dt = fixed_dts[cs];
    else if (P.dim == 1) dt = P.cfl * P.dx / sx;
    else dt = P.cfl / (sx / P.dx + sy / P.dy);
    const bool dt_ok = dt > 0.0 && isfinite(dt);
    if (!dt_ok) dt = 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      if (!dt_ok) atomicOr(&sc->status, ST_DT);
      sc->dt = dt;
      sc->Sx = sx;
      sc->Sy = sy;
      dtlog[cs] = dt;
      // the other parity's maxima were last read before the previous
      // step's second barrier: clear them for the next step
      atomicExch(&ps->smax[par ^ 1][0], 0ull);
      atomicExch(&ps->smax[par ^ 1][1], 0ull);
    }
    // B: cells
    double mh = 0.0, mz = 0.0;
    int cst = 0;
    for (long long k = t0; k < ncell; k += stride) {
      double a = 0.0, b = 0.0;
      cst |= cell_item(P, S, k, dt, a, b);
      mh += a;
      mz += b;
    }
    mh = warp_sum(mh);
    mz = warp_sum(mz);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cst |= __shfl_xor_sync(0xffffffffu, cst, o);
    if (threadIdx.x == 0) {
      if (cst) atomicOr(&sc->status, cst);
      mpart[2 * blockIdx.x] = mh;
      mpart[2 * blockIdx.x + 1] = mz;
    }
    if (!grid_barrier(ps, expected, gen, polls)) {
      if (threadIdx.x == 0) atomicOr(&sc->status, ST_SYNC);
      return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      sc->t += dt;
      sc->steps += 1;
      sc->call_step = cs + 1;
      sc->mass_parts = gridDim.x;
    }
  }
}

}  // namespace sve
