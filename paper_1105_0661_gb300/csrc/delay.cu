// Stand-alone sub-sample delay compensation + bandpass + corner turn (Sections 3 and 4.3):
//   ct[f][c][s][pol][m] = chan[f][s][pol][m][c] * bp[c] * exp(+2 pi i (f0_f tau_s + df_c (tau_s - n_s Ts)))
// The phase is formed in FP64 cycles per (s, f, c) and reduced before the FP32 sine/cosine; the
// transpose goes through an XOR-swizzled shared-memory tile so that both the 2 KB channel rows read
// and the 128-byte spectrum runs written are coalesced and bank-conflict free.
#include "lbf_internal.cuh"

namespace lbf {
namespace {

constexpr int kTile = 16;   // spectra per CTA

__global__ void __launch_bounds__(256)
delay_ct_kernel(Geometry g, const float2 *__restrict__ chan, float2 *__restrict__ ct, int tiles) {
  __shared__ __align__(16) float2 stage[kN * kTile];
  const int tid = threadIdx.x;
  long long idx = blockIdx.x;
  const int tile = (int)(idx % tiles);
  idx /= tiles;
  const int pol = (int)(idx % kP);
  idx /= kP;
  const int s = (int)(idx % g.S);
  const int f = (int)(idx / g.S);
  const int m0 = tile * kTile;

  const int c = tid;
  const double df = (double)(c - kN / 2) * (g.fs / kN);
  const double phi = g.f0[f] * g.tau[s] + df * g.resid[s];
  const float2 ph = unit_phasor_cycles(phi);
  const float b = g.bandpass[c];
  const float2 gain = make_float2(b * ph.x, b * ph.y);

  const float2 *src = chan + (((long long)f * g.S + s) * kP + pol) * g.M * kN;
#pragma unroll 4
  for (int q = 0; q < kTile; ++q) {
    const int m = m0 + q;
    if (m < g.M) stage[c * kTile + (q ^ (c & 15))] = cmul(src[(long long)m * kN + c], gain);
  }
  __syncthreads();
  const int q = tid & 15;
  if (m0 + q < g.M) {
#pragma unroll 4
    for (int pass = 0; pass < kN / 16; ++pass) {
      const int cc = pass * 16 + (tid >> 4);
      ct[((((long long)f * kN + cc) * g.S + s) * kP + pol) * g.M + m0 + q] =
          stage[cc * kTile + (q ^ (cc & 15))];
    }
  }
}

}  // namespace

cudaError_t launch_delay_ct(const Geometry &g, const float2 *chan, float2 *ct, cudaStream_t st) {
  const int tiles = (g.M + kTile - 1) / kTile;
  const long long ctas = (long long)g.F * g.S * kP * tiles;
  if (ctas == 0) return cudaSuccess;
  delay_ct_kernel<<<(unsigned)ctas, 256, 0, st>>>(g, chan, ct, tiles);
  return cudaGetLastError();
}

}  // namespace lbf
