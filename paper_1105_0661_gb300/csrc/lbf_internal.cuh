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
  int S, F, B, T, M, Q, nS;   // stations, subbands, beams, samples/block, spectra, int. factor, Stokes
  int H;                      // history samples per (station, subband)
  double fs;                  // subband sample rate
  const float *taps;          // [L*N]
  const float2 *twiddle;      // [N] exp(-2 pi i n / N)
  const float *bandpass;      // [N]
  const int *dshift;          // [S] integer shift d_s
  const double *tau;          // [S] phase-centre delay tau_s
  const double *resid;        // [S] tau_s - n_s Ts
  const double *f0;           // [F] subband centre frequency
  const double *dtau;         // [B][S] beam delay difference
};

enum OutKind { OUT_VOLTAGES = 0, OUT_STOKES_I = 1, OUT_STOKES_IQUV = 4 };

// --- launchers (return cudaGetLastError() of the launch) ---
// a1-a3 (+ a4 when ct != nullptr): filter bank; reads history `hist`, block `in`.
cudaError_t launch_ppf(const Geometry &g, int bits, const void *in, const void *hist,
                       float2 *chan, float2 *ct, cudaStream_t st);
// history update: new_hist = last H samples of [hist | in]
cudaError_t launch_hist_update(const Geometry &g, int bits, const void *in, const void *hist,
                               void *new_hist, cudaStream_t st);
// a4 standalone: chan -> ct
cudaError_t launch_delay_ct(const Geometry &g, const float2 *chan, float2 *ct, cudaStream_t st);
// a5-a6 (+ a7): beam former; out_kind selects voltages or fused Stokes; variant 1 few, 2 many
cudaError_t launch_beamform(const Geometry &g, int variant, int out_kind, const float2 *ct,
                            void *out, cudaStream_t st);
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

}  // namespace lbf
