// sve_handle.h -- the handle of libsve (private to the library's sources).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "../../include/sve.h"
#include "sve_device.cuh"
#include "sve_persist.cuh"
#include "sve_march.cuh"
#include "sve_split.cuh"

struct sve_adjoint_rec;  // recorded forward run (sve_adjoint.cu)

struct sve_handle {
  sve_config cfg;
  sve::DevParams P;
  int device = 0;
  cudaStream_t stream = nullptr;   // user stream (nullptr = legacy default)
  cudaStream_t capture = nullptr;  // private stream used only to capture graphs
  cudaStream_t upload = nullptr;   // private stream for host uploads in row chunks (overlapped with their projection)
  cudaEvent_t up_ev[5] = {};       // [0]: prior work of the handle's stream; [1..4]: the chunks
  double last_t = 0.0;             // simulated time read back with the status of the last blocking call
  bool has_state = false;
  size_t elem = 8;                 // bytes per state element
  long long next = 0;              // padded cells
  void* fields[13] = {};           // h hu hv z tau u v pi omx omy ca cbx cby
  void* fx = nullptr;
  void* fy = nullptr;
  double* mpart = nullptr;
  sve::DevScalars* sc = nullptr;
  double* dtlog = nullptr;
  int dtlog_cap = 0;
  double* fixed = nullptr;
  int fixed_cap = 0;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // [fixed]
  // FP32 state in 2D: the fused stencil (solve pass of strips marching over
  // rows, apply pass)
  bool fused = false;
  bool carry = false;          // fused, and no external sides: the carried update within a call
  void* alt[4] = {};           // second state buffer of the carried update (= fields[4..7], unused by this form)
  sve::MarchShape march = {};  // launch shape of the solve pass (sve_march.cuh)
  int agx = 0, agy = 0;    // apply pass grid (grid stride over columns and rows)
  int nt = 256;   // threads per block of the two-kernel step (32 or 256)
  int nsm = 152;  // SMs of the device
  // small grids: many steps per cooperative launch (sve_persist.cuh)
  sve::PersistScratch* ps = nullptr;
  int persist_mode = 0;    // 1: persistent launches when eligible (sve_set_persistent)
  bool persist_ok = false; // eligible: two-kernel form and the launch fits co-resident
  int pgrid = 0;           // one-warp blocks of the persistent launch
  int pmax = 0;            // most co-resident one-warp blocks allowed
  long long last_launches = 0;
  int last_steps = 0;
  // kernel timing (sve_profile): 3 events per step, read back lazily; per
  // triple, which of its two intervals count (bit 0: the solve pass, bit 1:
  // the update pass)
  bool profiling = false;
  std::vector<cudaEvent_t> events;
  std::vector<unsigned char> ev_kind;
  size_t events_used = 0;
  double prof_ms[2] = {0.0, 0.0};
  long long prof_launches[2] = {0, 0};
  // per-step history ring (sve_set_history): capacity records of 6 doubles
  double* hist = nullptr;
  int hist_cap = 0;
  // the splitting scheme (sve_split.cuh; FP64): 1 when on; the step's
  // parameters with the transport switched off; the held bed (padded)
  int scheme = 0;
  sve::DevParams P_sw;
  double* zsave = nullptr;
  sve_adjoint_rec* adj = nullptr;
  long long adj_budget = -1;  // bytes of forward data a recording may keep (-1: half the free device memory)
  void* halo = nullptr;    // staging of one side's ghost ring for the block calls (sve_block.cu)
};

// The handle's device arrays as a DevState of precision T.
template <typename T>
inline sve::DevState<T> state_of(const sve_handle* h) {
  sve::DevState<T> S;
  T** f[13] = {&S.h, &S.hu, &S.hv, &S.z, &S.tau, &S.u, &S.v, &S.pi, &S.omx, &S.omy, &S.ca, &S.cbx, &S.cby};
  for (int k = 0; k < 13; ++k) *f[k] = (T*)h->fields[k];
  S.fx = (T*)h->fx;
  S.fy = (T*)h->fy;
  return S;
}

// Implemented in sve_adjoint.cu: releases the recorded forward run.
__attribute__((visibility("hidden"))) void sve_internal_adjoint_free(sve_handle* h);
// Implemented in sve_api.cu: the time-step log holds >= n steps (the step
// graphs are rebuilt if it moves).
__attribute__((visibility("hidden"))) int sve_internal_reserve_dtlog(sve_handle* h, int n);
