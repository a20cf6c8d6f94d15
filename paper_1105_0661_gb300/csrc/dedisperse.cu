// Channel-level dedispersion (Section 4.4) of tied-array beam voltages.
//
// Dispersion in the interstellar medium delays lower frequencies; inside one channel the delay
// varies with the offset nu from the channel's sky frequency f_c.  Every run of K consecutive
// spectra of a (beam, subband, channel, pol) series is transformed by a K-point FFT into
// sub-channels of width (fs/N)/K, multiplied by the coherent-dedispersion chirp
//     H(nu) = exp(-2 pi i K_DM DM nu^2 / (f_c^2 (f_c + nu)))
// (the conjugate of the medium's transfer function, Hankins & Rickett 1975; K_DM is the constant of
// the cold-plasma delay law t = K_DM DM / f^2) and transformed back.  Runs do not overlap.
//
// One CTA serves one (subband, channel) and a group of 8 beams, which share the chirp.  Run length
// 256 (the default: 3 Hz sub-channels) uses the filter bank's 16 x 16 register FFT; any other
// power of two builds the twiddle table exp(-2 pi i n / K) and the chirp (at bit-reversed
// positions, scaled by 1/K) in shared memory once, then for each beam loads the 2 pols x M/K runs
// (contiguous in the voltage layout) in passes, runs an in-place radix-2 decimation-in-frequency
// FFT (natural order in, bit-reversed out), multiplies by the chirp, and runs the inverse as
// decimation in time (bit-reversed in, natural out), so no reordering pass is needed.  FP32
// throughout except the chirp phase, whose large term is reduced exactly in 64-bit fixed point.
#include "fft16.cuh"
#include "lbf_internal.cuh"

namespace lbf {
namespace {

constexpr int kThreads = 256;
constexpr int kBeamsPerCta = 8;
constexpr double kKdm = 4.148808e15;     // s Hz^2 per (pc cm^-3): cold-plasma delay t = kKdm DM / f^2
constexpr int kDataFloat2 = 8192;        // shared data per pass: 64 KB of complex samples

struct DdParams {
  int K, logK, runs, runs_per_pass;      // runs = 2 M / K per (beam, subband, channel)
  double dm;
};

// Per-channel chirp coefficients.  With nu = j' r (r = (fs/N)/K the sub-channel width, j' the
// signed bin) the chirp phase is
//     phi(j') = C j'^2 / (1 + eps j'),  C = K_DM DM r^2 / f_c^3,  eps = r / f_c,
// which can reach thousands of cycles, so it is split exactly: phi = C j'^2 - C eps j'^3/(1 + eps j').
// The first term is reduced modulo one in 64-bit fixed point (frac(C) j'^2 mod 2^64, exact); the
// second, at most phi eps |j'| (eps |j'| <= (fs/N/2)/f_c), is small enough for FP32.
struct ChirpCoef {
  unsigned long long frac;   // frac(C) in units of 2^-64 cycle
  float c, eps;
};

__device__ __forceinline__ ChirpCoef chirp_coef(const Geometry &g, int f, int c, int K, double dm) {
  const double f_c = g.f0[f] + (double)(c - kN / 2) * (g.fs / kN);
  const double r = g.fs / kN / (double)K;
  const double C = kKdm * dm * r * r / (f_c * f_c * f_c);
  ChirpCoef k;
  k.frac = (unsigned long long)ldexp(C - floor(C), 64);
  k.c = (float)C;
  k.eps = (float)(r / f_c);
  return k;
}

// exp(-2 pi i phi(j')) / K for the signed bin j'
__device__ __forceinline__ float2 chirp_value(const ChirpCoef &k, int jj, float scale) {
  const unsigned long long sq = (unsigned long long)((long long)jj * jj);
  const float main = (float)(long long)(k.frac * sq) * 5.421010862427522e-20f;   // x 2^-64: [-1/2, 1/2)
  const float fj = (float)jj, a = k.eps * fj;
  float ph = main - k.c * fj * fj * a / (1.0f + a);   // cycles
  ph -= rintf(ph);
  float s, co;
  sincospif(2.0f * ph, &s, &co);
  return make_float2(co * scale, -s * scale);
}

__global__ void __launch_bounds__(kThreads)
dedisperse_kernel(Geometry g, DdParams d, const float2 *in, float2 *out) {   // in may equal out
  extern __shared__ __align__(16) float2 sm[];
  const int K = d.K, half = K >> 1;
  float2 *x = sm;                              // [runs_per_pass][K] (16-byte aligned: float4 copies)
  float2 *tw = x + d.runs_per_pass * K;        // [K/2]  exp(-2 pi i n / K)
  float2 *chirp = tw + half;                   // [K]    H(nu_j) / K at position bitrev(j)
  __shared__ ChirpCoef coef_s;

  const int bgroups = (g.B + kBeamsPerCta - 1) / kBeamsPerCta;
  const long long fc = blockIdx.x / bgroups;
  const int bg = (int)(blockIdx.x - fc * bgroups);
  const int f = (int)(fc / kN), c = (int)(fc - (long long)f * kN);
  const int tid = threadIdx.x;

  if (tid == 0) coef_s = chirp_coef(g, f, c, K, d.dm);
  for (int n = tid; n < half; n += kThreads) {
    float s, co;
    sincospif(2.0f * (float)n / (float)K, &s, &co);
    tw[n] = make_float2(co, -s);
  }
  __syncthreads();
  const float scale = 1.0f / (float)K;
  for (int i = tid; i < K; i += kThreads) {
    const int j = (int)(__brev((unsigned)i) >> (32 - d.logK));   // FFT bin held at position i
    chirp[i] = chirp_value(coef_s, j < half ? j : j - K, scale);
  }
  __syncthreads();

  const int b_end = min(g.B, (bg + 1) * kBeamsPerCta);
  for (int b = bg * kBeamsPerCta; b < b_end; ++b) {
    const long long base = (((long long)b * g.F + f) * kN + c) * (long long)kP * g.M;   // [P][M] of (b, f, c)
    for (int r0 = 0; r0 < d.runs; r0 += d.runs_per_pass) {
      const int nr = min(d.runs_per_pass, d.runs - r0);
      const int n = nr * K;
      const float4 *src = reinterpret_cast<const float4 *>(in + base + (long long)r0 * K);
      for (int i = tid; i < n / 2; i += kThreads) reinterpret_cast<float4 *>(x)[i] = src[i];
      __syncthreads();
      // forward FFT, decimation in frequency: stage size L = K .. 2
      for (int hl = half; hl >= 1; hl >>= 1) {
        const int lhl = __ffs(hl) - 1;
        const int stride = half >> lhl;            // twiddle index step K / L
        for (int u = tid; u < nr * half; u += kThreads) {
          const int run = u >> (d.logK - 1), t_all = u & (half - 1);
          const int grp = t_all >> lhl, t = t_all & (hl - 1);
          float2 *p0 = x + run * K + grp * 2 * hl + t;
          const float2 a = p0[0], bb = p0[hl];
          p0[0] = make_float2(a.x + bb.x, a.y + bb.y);
          p0[hl] = cmul(make_float2(a.x - bb.x, a.y - bb.y), tw[t * stride]);
        }
        __syncthreads();
      }
      for (int i = tid; i < n; i += kThreads) x[i] = cmul(x[i], chirp[i & (K - 1)]);
      __syncthreads();
      // inverse FFT, decimation in time: stage size L = 2 .. K, conjugate twiddles
      for (int hl = 1; hl <= half; hl <<= 1) {
        const int lhl = __ffs(hl) - 1;
        const int stride = half >> lhl;
        for (int u = tid; u < nr * half; u += kThreads) {
          const int run = u >> (d.logK - 1), t_all = u & (half - 1);
          const int grp = t_all >> lhl, t = t_all & (hl - 1);
          float2 *p0 = x + run * K + grp * 2 * hl + t;
          const float2 w = tw[t * stride];
          const float2 a = p0[0], bw = cmul(p0[hl], make_float2(w.x, -w.y));
          p0[0] = make_float2(a.x + bw.x, a.y + bw.y);
          p0[hl] = make_float2(a.x - bw.x, a.y - bw.y);
        }
        __syncthreads();
      }
      float4 *dst = reinterpret_cast<float4 *>(out + base + (long long)r0 * K);
      for (int i = tid; i < n / 2; i += kThreads) dst[i] = reinterpret_cast<const float4 *>(x)[i];
      __syncthreads();
    }
  }
}

// K = 256 (sub-channels of (fs/N)/256 = 3 Hz): the filter bank's 16 x 16 decomposition in
// registers, one transform per 16-thread group at a time.  Each group streams its own transforms:
// thread j loads x[16 p1 + j] straight from global memory (a half-warp reads 128 contiguous bytes
// per load), transposes once through its shared row (rows of 16 padded to 17, so both walks are
// conflict-free with fixed offsets), and ends holding bins j + 16 k2.  Those are exactly the
// inputs x[16 p1 + j], p1 = k2, of its next transform, so it multiplies them by the chirp,
// conjugates, and runs the same forward transform again in registers (the inverse is
// conj(FFT(conj(.)))), then stores y[j + 16 k2] straight to global memory.  Groups synchronise
// only among their own 16 lanes.
__global__ void __launch_bounds__(kThreads, 3)   // 3 CTAs per SM: more transforms' loads in flight
dedisperse256_kernel(Geometry g, DdParams d, const float2 *in, float2 *out) {   // in may equal out
  constexpr int K = 256;
  __shared__ float2 x[16][16 * 17];            // one padded row per 16-thread group
  __shared__ float2 tw[K];                     // [k1][j] = exp(-2 pi i j k1 / 256)
  __shared__ float2 chirp[K];                  // natural bin order, scaled by 1/256
  __shared__ ChirpCoef coef_s;
  const int bgroups = (g.B + kBeamsPerCta - 1) / kBeamsPerCta;
  const long long fc = blockIdx.x / bgroups;
  const int bg = (int)(blockIdx.x - fc * bgroups);
  const int f = (int)(fc / kN), c = (int)(fc - (long long)f * kN);
  const int tid = threadIdx.x, j = tid & 15, grp = tid >> 4;
  const unsigned mask = 0xFFFFu << (16 * (grp & 1));   // this group's lanes of the warp
  if (tid == 0) coef_s = chirp_coef(g, f, c, K, d.dm);
  {
    float s, co;
    sincospif(2.0f * (float)((tid & 15) * (tid >> 4)) / (float)K, &s, &co);
    tw[tid] = make_float2(co, -s);
  }
  __syncthreads();
  chirp[tid] = chirp_value(coef_s, tid < K / 2 ? tid : tid - K, 1.0f / (float)K);
  __syncthreads();

  float2 *r = x[grp];
  // rest of the forward transform from a[p1] = x[16 p1 + j]: thread j ends with X[j + 16 k2]
  auto fft_tail = [&](float2 (&a)[16]) {
    dft16(a);
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) r[17 * k1 + j] = cmul(a[k1], tw[16 * k1 + j]);
    __syncwarp(mask);
#pragma unroll
    for (int p2 = 0; p2 < 16; ++p2) a[p2] = r[17 * j + p2];
    __syncwarp(mask);   // the row is rewritten by the next transform
    dft16(a);
  };
  const int b0 = bg * kBeamsPerCta;
  const int ntr = (min(g.B, b0 + kBeamsPerCta) - b0) * d.runs;   // transforms of this CTA
  for (int tr = grp; tr < ntr; tr += 16) {
    const int b = b0 + tr / d.runs, run = tr % d.runs;
    const long long off = (((long long)b * g.F + f) * kN + c) * (long long)kP * g.M + (long long)run * K;
    float2 a[16];
#pragma unroll
    for (int p1 = 0; p1 < 16; ++p1) a[p1] = in[off + 16 * p1 + j];
    fft_tail(a);
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) {     // chirp (with 1/256), then conjugate for the inverse
      const float2 v = cmul(a[k2], chirp[j + 16 * k2]);
      a[k2] = make_float2(v.x, -v.y);
    }
    fft_tail(a);
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) out[off + j + 16 * k2] = make_float2(a[k2].x, -a[k2].y);
  }
}

}  // namespace

cudaError_t launch_dedisperse(const Geometry &g, double dm, int K, const float2 *in, float2 *out, cudaStream_t st) {
  if (g.M == 0 || g.B == 0) return cudaSuccess;
  DdParams d;
  d.K = K;
  d.logK = 0;
  while ((1 << d.logK) < K) ++d.logK;
  d.runs = kP * g.M / K;
  d.runs_per_pass = kDataFloat2 / K < d.runs ? kDataFloat2 / K : d.runs;
  if (d.runs_per_pass < 1) d.runs_per_pass = 1;
  d.dm = dm;
  const long long ctas = (long long)g.F * kN * ((g.B + kBeamsPerCta - 1) / kBeamsPerCta);
  if (K == 256) {
    dedisperse256_kernel<<<(unsigned)ctas, kThreads, 0, st>>>(g, d, in, out);
    return cudaGetLastError();
  }
  const size_t smem = sizeof(float2) * ((size_t)K / 2 + K + (size_t)d.runs_per_pass * K);
  cudaError_t e = cudaFuncSetAttribute(dedisperse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dedisperse_kernel<<<(unsigned)ctas, kThreads, smem, st>>>(g, d, in, out);
  return cudaGetLastError();
}

}  // namespace lbf
