// Stand-alone sub-sample delay compensation + bandpass + corner turn (Sections 3 and 4.3):
//   ct[f][c][s][pol][m] = chan[f][s][pol][m][c] * bp[c] * exp(+2 pi i (f0_f tau_s + df_c (tau_s - n_s Ts)))
// The phase is formed in FP64 cycles per (s, f, c) and reduced before the FP32 sine/cosine; the
// transpose goes through an XOR-swizzled shared-memory tile so that both the 2 KB channel rows read
// and the 128-byte spectrum runs written are coalesced and bank-conflict free.
#include <cuda_fp16.h>

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

// ct [F][N][S][P][M] cf32 -> [F][N][P][M][kpad] fp16 planes (station slot 2s, 2s+1).  One CTA per
// (f, c, pol, 64-spectrum tile): stations are gathered through shared memory so that each thread
// writes one whole 4-station (16-byte) group of a spectrum's row.
__global__ void __launch_bounds__(256)
ct_to_ct16_kernel(Geometry g, const float2 *__restrict__ ct, Ct16Out o, int tiles) {
  __shared__ float2 tile[64][65];
  long long idx = blockIdx.x;
  const int t = (int)(idx % tiles);
  idx /= tiles;
  const int pol = (int)(idx % kP);
  const long long fc = idx / kP;
  const int m0 = t * 64;
  __half *hi = reinterpret_cast<__half *>(o.hi);
  __half *lo = reinterpret_cast<__half *>(o.lo);
  for (int s0 = 0; s0 < g.S; s0 += 64) {
    __syncthreads();
    for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) {
      const int sl = i >> 6, ml = i & 63, s = s0 + sl, m = m0 + ml;
      tile[ml][sl] = (s < g.S && m < g.M) ? ct[((fc * g.S + s) * kP + pol) * g.M + m] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) {
      const int ml = i >> 6, sl = i & 63, s = s0 + sl, m = m0 + ml;
      if (s < g.S && m < g.M) {
        const float2 v = tile[ml][sl];
        const long long d = (((fc * kP + pol) * g.M) + m) * o.kpad + 2 * s;
        const __half2 h = __floats2half2_rn(v.x, v.y);
        *reinterpret_cast<__half2 *>(hi + d) = h;
        if (lo) *reinterpret_cast<__half2 *>(lo + d) = __floats2half2_rn(v.x - __low2float(h), v.y - __high2float(h));
      }
    }
  }
}

}  // namespace

cudaError_t launch_ct_to_ct16(const Geometry &g, const float2 *ct, const Ct16Out &o, cudaStream_t st) {
  const int tiles = (g.M + 63) / 64;
  const long long ctas = (long long)g.F * kN * kP * tiles;
  if (ctas == 0) return cudaSuccess;
  ct_to_ct16_kernel<<<(unsigned)ctas, 256, 0, st>>>(g, ct, o, tiles);
  return cudaGetLastError();
}

cudaError_t launch_delay_ct(const Geometry &g, const float2 *chan, float2 *ct, cudaStream_t st) {
  const int tiles = (g.M + kTile - 1) / kTile;
  const long long ctas = (long long)g.F * g.S * kP * tiles;
  if (ctas == 0) return cudaSuccess;
  delay_ct_kernel<<<(unsigned)ctas, 256, 0, st>>>(g, chan, ct, tiles);
  return cudaGetLastError();
}

}  // namespace lbf
