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

// ct [F][N][S][P][M] cf32 -> FP16 planes [F*N][kpad][Mb][P][32] (rows k = 2s re, 2s+1 im): an
// elementwise split, both sides spectrum-fastest, so reads and writes are coalesced as they are.
__global__ void __launch_bounds__(256)
ct_to_ct16_kernel(Geometry g, const float2 *__restrict__ ct, Ct16Out o, long long n) {
  __half *hi = reinterpret_cast<__half *>(o.hi);
  __half *lo = reinterpret_cast<__half *>(o.lo);
  const int mb = (g.M + 31) >> 5;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(i % g.M);
    const long long r = i / g.M;                             // (fc * S + s) * P + pol
    const int pol = (int)(r % kP);
    const long long fcs = r / kP;
    const long long fc = fcs / g.S;
    const int s = (int)(fcs - fc * g.S);
    const float2 v = ct[i];
    const long long re = (((fc * o.kpad + 2 * s) * mb + (m >> 5)) * 64) + pol * 32 + (m & 31);
    const long long im = re + (long long)mb * 64;
    const __half hr = __float2half_rn(v.x), hm = __float2half_rn(v.y);
    hi[re] = hr;
    hi[im] = hm;
    if (lo) {
      lo[re] = __float2half_rn(v.x - __half2float(hr));
      lo[im] = __float2half_rn(v.y - __half2float(hm));
    }
  }
}

}  // namespace

cudaError_t launch_ct_to_ct16(const Geometry &g, const float2 *ct, const Ct16Out &o, cudaStream_t st) {
  const long long n = (long long)g.F * kN * g.S * kP * g.M;
  if (n == 0) return cudaSuccess;
  const long long want = (n + 255) / 256;
  ct_to_ct16_kernel<<<(unsigned)(want < 152LL * 64 ? want : 152LL * 64), 256, 0, st>>>(g, ct, o, n);
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
