// Plan-time device tables for the positional weights (Section 4.3) in FP64.
//
// The weight phase of beam b, station s in channel c of subband f is, in cycles,
//     phi = f_c * dtau[b,s] = f0_f * dtau[b,s] + (c - N/2) * df * dtau[b,s],
// with |(c - N/2) df dtau| well below one cycle for any tied-array beam inside a station beam.
// The large carrier term is formed and reduced to [-1/2, 1/2] cycle here, in FP64, once per
// (subband, beam, station); the beam formers then add the small per-channel term in FP32 and take
// an FP32 sincos.  The reduced value is exact to FP32 rounding (<= 3e-8 cycle), the channel term
// to < 1e-7 cycle, so a weight is accurate to ~1e-6 relative -- without any per-sample FP64 work.
#include "lbf_internal.cuh"

namespace lbf {
namespace {

// With tau and resid given, station s's delay compensation (Sections 3, 4.3) is folded in: the
// phase of Y_s = X_s exp(+2 pi i (f0_f tau_s + df_c (tau_s - n_s Ts))) has the same form (a
// subband term plus (c - N/2) times a per-channel step), so w Y_s = w' X_s with the tables of
// dtau[b,s] + tau_s and dtau[b,s] + resid_s.
__global__ void phase_table_kernel(int F, int B, int S, double fs, const double *__restrict__ f0,
                                   const double *__restrict__ dtau, const double *__restrict__ tau,
                                   const double *__restrict__ resid, float *__restrict__ phase0,
                                   float *__restrict__ step) {
  const long long n = (long long)F * B * S;
  const double df = fs / kN;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long bs = i % ((long long)B * S);
    const int f = (int)(i / ((long long)B * S));
    const int s = (int)(bs % S);
    const double phi = f0[f] * (dtau[bs] + (tau ? tau[s] : 0.0));
    phase0[i] = (float)(phi - rint(phi));
    if (f == 0) step[bs] = (float)(df * (dtau[bs] + (resid ? resid[s] : 0.0)));
  }
}

}  // namespace

cudaError_t launch_phase_tables(int F, int B, int S, double fs, const double *f0, const double *dtau,
                                float *phase0, float *step, cudaStream_t st, const double *tau,
                                const double *resid) {
  const long long n = (long long)F * B * S;
  if (n == 0) return cudaSuccess;
  const long long want = (n + 255) / 256;
  phase_table_kernel<<<(unsigned)(want < 4096 ? want : 4096), 256, 0, st>>>(F, B, S, fs, f0, dtau, tau, resid,
                                                                             phase0, step);
  return cudaGetLastError();
}

}  // namespace lbf
