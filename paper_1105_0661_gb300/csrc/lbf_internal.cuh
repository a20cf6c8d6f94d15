// Internal declarations shared by the kernels and the C-ABI layer of the LOFAR beam-former library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbf {

constexpr int kN = 256;   // channels per subband (256-point FFT)
constexpr int kL = 16;    // FIR taps per channel
constexpr int kP = 2;     // polarisations X, Y

// Device-side description of one observation; every pointer is device memory owned by the plan.
struct Geometry {
  int S = 0, F = 0, B = 0, T = 0, M = 0, Q = 1, nS = 0;   // stations, subbands, beams, samples/block,
                                                        // spectra, integration factor, Stokes
  int H = 0;                  // history samples per (station, subband)
  int inc = 0;                // 1: the Stokes output also holds the incoherent beam at index B
  int tc_wlo = 1;             // tensor-core beam former: 1 adds the Wlo Yhi product (three
                              // products), 0 keeps FP16 weights only (two products)
  double fs = 0.0;            // subband sample rate
  const float *taps = nullptr;          // [L*N]
  const float2 *twiddle = nullptr;      // [N] exp(-2 pi i n / N)
  const float *bandpass = nullptr;      // [N]
  const int *dshift = nullptr;          // [S] integer shift d_s
  const double *tau = nullptr;          // [S] phase-centre delay tau_s
  const double *resid = nullptr;        // [S] tau_s - n_s Ts
  const double *f0 = nullptr;           // [F] subband centre frequency
  const double *dtau = nullptr;         // [B][S] beam delay difference
  const float *phase0 = nullptr;        // [F][B][S] f0_f dtau[b,s] reduced to [-1/2, 1/2] cycle (FP64 -> FP32)
  const float *step = nullptr;          // [B][S] fs/N * dtau[b,s], cycles per channel
  // the same two tables with the delay compensation folded in (tensor-core plans): phase
  // f0_f (dtau[b,s] + tau_s) reduced, step fs/N (dtau[b,s] + tau_s - n_s Ts)
  const float *phase0g = nullptr;
  const float *stepg = nullptr;
  int ct16_raw = 0;           // 1: the FP16 planes hold the filtered spectrum before the delay phase
                              // and bandpass, which the tensor-core weights then carry
  int *err = nullptr;                   // device error word: a bounded wait that gave up records here
  long long ppf_stall = -1;             // failure-detection test: this filter-bank CTA issues no input copies
};

// Codes of the device error word (lbf_device_status): the role whose bounded wait expired.
// DERR_PPF_ALIGN is not a wait: the filter bank's shared memory was not 128-byte aligned for its
// tensor stores, and it wrote nothing.
enum DeviceErr { DERR_NONE = 0, DERR_TC_LOADS = 1, DERR_TC_MMA = 2, DERR_TC_EPILOGUE = 3, DERR_PPF_INPUT = 4,
                 DERR_PPF_ALIGN = 5 };

enum OutKind { OUT_VOLTAGES = 0, OUT_STOKES_I = 1, OUT_STOKES_IQUV = 4 };

// FP16 corner-turned scratch of the tensor-core beam former: [F*N][Mt][kpad][P][32] halves per
// plane (k = 2 station + re|im; tiles of 32 spectra, the two pols side by side), Mt = tc_tiles(M)
// an even count so that the beam former reads tiles in pairs.
struct Ct16Out {
  void *hi, *lo;   // lo may be null (single-product form)
  int kpad;        // 2 S rounded up to a multiple of 16
};
__host__ __device__ inline int tc_tiles(int M) { return ((M + 63) / 64) * 2; }
// Tensor map (CUtensorMap, 128 bytes, written to `map`) of one FP16 plane at `base` for the filter
// bank's tensor stores: boxes of 16 spectra of one pol x 2 K rows x 256 channels, no swizzle.
cudaError_t encode_ct16_store_map(void *map, void *base, int kpad, int M, long long fc_rows);
// The same for the FP32 corner turn [F*N][S][P][M] float2 (M even): boxes of 16 spectra of one
// (station, pol) x `nch` consecutive channels.
cudaError_t encode_ct32_store_map(void *map, void *base, int S, int M, long long fc_rows, int nch);

// One observation of a batch (grouped persistent launches, batch.cu): its geometry, this
// block's buffers, and its range of work items in the grouped filter bank and beam former.
struct PpfGroup {
  Geometry g;
  const void *in;
  const void *hist;
  void *new_hist;
  float2 *ct;                 // corner-turned scratch of this observation (FP32 plans)
  Ct16Out ct16;               // FP16 hi+lo planes (tensor-core plans)
  int tc;                     // 1: write ct16 instead of ct
  int bits;
  int spc;                    // spectra per filter-bank work item (a multiple of 16; both pols)
  int chunks;                 // ceil(M / spc)
  long long first_item;       // first filter-bank work item of this group
  long long first_hist;       // first history element of this group
  const void *maps;           // device copy of its output's tensor maps (ppf_group_maps), when
                              // the group is in a tensor-store launch class
};
struct BfGroup {
  Geometry g;
  const float2 *ct;
  void *out;
  int variant;                // 1 few-beam, 2 many-beam (128-beam tiles), 3 many-beam (64-beam tiles)
  int out_kind;
  int per_fc;                 // work items per (subband, channel): beam groups or beam tiles
  long long first_item;
};

// --- launchers (return cudaGetLastError() of the launch) ---
// a1-a3 (+ a4 when ct or ct16 is given): filter bank; reads history `hist`, block `in`.
cudaError_t launch_ppf(const Geometry &g, int bits, const void *in, const void *hist,
                       float2 *chan, float2 *ct, cudaStream_t st, const Ct16Out *ct16 = nullptr);
// batch: persistent grouped filter bank (FP32 corner-turned output), history update, beam former.
// A grouped launch takes its groups (HOST array, at most kMaxGroups) as a grid-constant kernel
// parameter, so that a work item reads its observation's geometry from the constant bank, as a
// kernel of one observation does.
constexpr int kMaxGroups = 64;
struct PpfTable { PpfGroup grp[kMaxGroups]; int n; };
struct BfTable { BfGroup grp[kMaxGroups]; int n; };
// a kernel's parameters (the table, a count and a counter pointer) must fit in 32764 bytes
static_assert(sizeof(PpfTable) + 16 <= 32764 && sizeof(BfTable) + 16 <= 32764, "grouped launch table too large");
// The group of work item `item` in a grouped launch: the last group whose first item is <= item
// (binary search, by one thread per item; the others read the result from shared memory).
template <class Table>
__device__ __forceinline__ int group_of(const Table &T, long long item) {
  int lo = 0, hi = T.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (T.grp[mid].first_item <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}
// one persistent launch for the groups of one sample width and output form (FP32 corner turn or
// FP16 planes); items numbered from 0 within the launch
// Tensor-store output of a group's filter bank: whether its output allows it (FP16 planes always;
// the FP32 corner turn for even M), and the bytes and host encoding of its tensor maps, which the
// caller copies to device memory and points G.maps at.
bool ppf_group_tma(const PpfGroup &G);
size_t ppf_group_maps_bytes();
cudaError_t ppf_group_maps(const PpfGroup &G, void *host_dst);
cudaError_t launch_ppf_group(int bits, int tc, int tma, const PpfGroup *h_groups, int ngrp, long long total,
                             unsigned long long *counter, int ctas, cudaStream_t st);
// history update of all groups (DEVICE table: each thread looks up its own element's group)
cudaError_t launch_hist_group(const PpfGroup *d_groups, int ngrp, long long total, cudaStream_t st);
// filter-bank work items (both polarisations of one stream chunk) per (station, subband) stream
int ppf_items_per_stream(int M, int spc);
int ppf_ctas_per_sm();
// one persistent launch for groups of one beam-former variant (1, 2 or 3) and output kind, sized to
// the residency of that kernel with `smem` bytes of shared memory (bf_group_residency)
cudaError_t launch_bf_group(int variant, int out_kind, const BfGroup *h_groups, int ngrp, long long total,
                            unsigned long long *counter, size_t smem, cudaStream_t st);
int bf_group_residency(int variant, int out_kind, size_t smem);
int few_beams_per_item();
int many_beams_per_item(int variant);   // 128 (variant 2) or 64 (variant 3)
// AUTO beam-former choice: 1 few-beam, 2 many-beam 128-beam tiles, 3 many-beam 64-beam tiles
int auto_bf_variant(int B, int S);
size_t bf_smem_bytes(int variant, int S);
// FP32 corner-turned [F][N][S][P][M] -> FP16 [F][N][P][M][kpad] hi/lo planes (split-call TC path)
cudaError_t launch_ct_to_ct16(const Geometry &g, const float2 *ct, const Ct16Out &o, cudaStream_t st);
// superstation beam former: sum of delay-compensated stations per group (delay.cu)
cudaError_t launch_superstation(const Geometry &g, const float2 *ct, float2 *ss, const int *members, const int *offs,
                                int ngroups, cudaStream_t st);
// incoherent beam (index B of the Stokes output) from the FP16 planes of a tensor-core plan
cudaError_t launch_incoherent_ct16(const Geometry &g, int out_kind, const Ct16Out &o, float *out, cudaStream_t st);
// tcgen05 beam former with fused Stokes epilogue (bf_tc.cu); tm_hi/tm_lo are CUtensorMap*
// stall_item >= 0: failure-detection test, the loads of that work item are never issued
cudaError_t launch_bf_tc(const Geometry &g, int out_kind, const void *tm_hi, const void *tm_lo, float *out, int *err,
                         cudaStream_t st, long long stall_item = -1);
// several tensor-core plans of one output kind and integration length in ONE persistent launch
// (their work items numbered one after the other); n <= tc_max_plans_per_launch()
struct TcPlanRef {
  Geometry g;
  const void *tm_hi, *tm_lo;   // CUtensorMap* of the plan's FP16 planes
  float *out;
  int *err;
};
cudaError_t launch_bf_tc_group(const TcPlanRef *plans, int n, int out_kind, int Q, cudaStream_t st);
int tc_max_plans_per_launch();
// channel-level dedispersion of vol [B][F][N][P][M] (in may equal out); K a power of two dividing M
cudaError_t launch_dedisperse(const Geometry &g, double dm, int K, const float2 *in, float2 *out, cudaStream_t st);
int tc_max_stations();
int tc_spectra_per_tile();   // TMA box height of the FP16 scratch (spectra per N tile)
int tc_kpad(int S);
// history update: new_hist = last H samples of [hist | in]
cudaError_t launch_hist_update(const Geometry &g, int bits, const void *in, const void *hist,
                               void *new_hist, cudaStream_t st);
// a4 standalone: chan -> ct
cudaError_t launch_delay_ct(const Geometry &g, const float2 *chan, float2 *ct, cudaStream_t st);
// a5-a6 (+ a7): beam former; out_kind selects voltages or fused Stokes; variant 1 few, 2 many
// (128-beam tiles), 3 many (64-beam tiles)
cudaError_t launch_beamform(const Geometry &g, int variant, int out_kind, const float2 *ct,
                            void *out, cudaStream_t st);
// plan-time FP64 tables of the weight phases (tables.cu)
cudaError_t launch_phase_tables(int F, int B, int S, double fs, const double *f0, const double *dtau,
                                float *phase0, float *step, cudaStream_t st, const double *tau = nullptr,
                                const double *resid = nullptr);
// largest S the many-beam kernel accepts (shared-memory bound)
int many_beam_max_stations();
// a7 standalone: vol -> Stokes
cudaError_t launch_stokes(const Geometry &g, int out_kind, const float2 *vol, float *out,
                          cudaStream_t st);

// Shared device helpers --------------------------------------------------------------------------
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// exp(2 pi i phi) for a phase phi given in cycles (FP64): the phase is reduced to [-1/2, 1/2]
// cycle in FP64 before the FP32 sine/cosine, so large f*tau products keep full accuracy.
__device__ __forceinline__ float2 unit_phasor_cycles(double phi) {
  const double r = phi - rint(phi);
  float s, c;
  sincospif(2.0f * (float)r, &s, &c);
  return make_float2(c, s);
}

// Weight w[b,s] of channel c (Section 4.3) from the plan's phase tables: the FP64-reduced carrier
// phase of (f, b, s) plus the FP32 channel term, through an FP32 sincos.
__device__ __forceinline__ float2 beam_weight(const Geometry &g, int f, int c, long long bs) {
  const float phi = fmaf((float)(c - kN / 2), g.step[bs], g.phase0[(long long)f * g.B * g.S + bs]);
  float s, co;
  sincospif(2.0f * phi, &s, &co);
  return make_float2(co, s);
}

}  // namespace lbf
