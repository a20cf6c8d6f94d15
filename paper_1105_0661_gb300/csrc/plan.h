// Internal definition of a plan (lbf_plan_t), shared by the C-ABI layer and the batch runtime.
#pragma once

#include <cuda.h>

#include <vector>

#include "lbf.h"
#include "lbf_internal.cuh"

namespace lbf {
constexpr uint32_t kPlanMagic = 0x4c424650u;   // "LBFP"
}

struct lbf_plan_s {
  uint32_t magic = lbf::kPlanMagic;
  int device = 0;
  int S = 0, F = 0, N = 0, L = 0, B = 0, T = 0, M = 0, Q = 1, nS = 0, bits = 16;
  int out_kind = 0, variant = 1, d_max = 0, H = 0;
  double fs = 0.0;
  std::vector<int32_t> n_shift, d_shift;
  float *taps = nullptr;
  float2 *twiddle = nullptr;
  float *bandpass = nullptr;
  int *dshift = nullptr;
  double *tau = nullptr, *resid = nullptr, *f0 = nullptr, *dtau = nullptr;
  float *phase0 = nullptr, *step = nullptr;
  float *phase0g = nullptr, *stepg = nullptr;   // with the delay folded in (tensor-core plans)
  // tensor-core precision: FP16 corner-turned planes and their TMA descriptors
  bool tc = false;
  int tc_wlo = 1;               // three products (LBF_FP16_TC) or two (LBF_FP16_TC2)
  int kpad = 0, planes = 0;
  void *ct16[2] = {nullptr, nullptr};
  alignas(64) CUtensorMap tmap[2];
  size_t ct16_bytes = 0;
  bool external_ws = false;     // scratch passed per call (lbf_run_block_ws)
  int inc = 0;                  // 1: Stokes output holds the incoherent beam at index B
  int *ss_members = nullptr;    // [S] stations grouped for the superstation beam former
  int *ss_offs = nullptr;       // [S + 1] group offsets into ss_members
  size_t ws_need = 0;           // scratch bytes one block needs
  int *d_err = nullptr;   // device error word set by bounded waits that gave up
  long long stall_item = -1;   // lbf_debug_stall_next: one-shot, consumed by the next tensor-core launch
  void *hist[2] = {nullptr, nullptr};
  int cur = 0;
  float2 *ws = nullptr;
  size_t word = 8, hist_bytes = 0, ws_bytes = 0;

  // lbf_run_block_host: copy streams and the events that order them against the kernels
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaEvent_t ev_in_free = nullptr, ev_in_ready = nullptr, ev_out_ready = nullptr, ev_out_done = nullptr;
  // lbf_run_blocks_host: the plan's compute stream, its start event and one input-free event per
  // device input buffer (the two alternate)
  cudaStream_t cs = nullptr;
  cudaEvent_t ev_start = nullptr, ev_in_free2[2] = {nullptr, nullptr};

  // kernel timing trace (lbf_trace_begin / lbf_trace_end)
  struct TraceSlot { int kernel; cudaEvent_t a, b; };
  std::vector<TraceSlot> trace;
  size_t trace_used = 0;
  int trace_dropped = 0;
  bool tracing = false;

  lbf::Geometry geometry() const {
    lbf::Geometry g;
    g.S = S; g.F = F; g.B = B; g.T = T; g.M = M; g.Q = Q; g.nS = nS; g.H = H; g.fs = fs;
    g.taps = taps; g.twiddle = twiddle; g.bandpass = bandpass; g.dshift = dshift;
    g.tau = tau; g.resid = resid; g.f0 = f0; g.dtau = dtau; g.phase0 = phase0; g.step = step;
    g.phase0g = phase0g; g.stepg = stepg;
    g.inc = inc;
    g.tc_wlo = tc_wlo;
    g.err = d_err;
    return g;
  }
};

