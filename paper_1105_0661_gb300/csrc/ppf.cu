// Poly-phase filter bank of Section 4.2: integer sample shift (Section 3), int->float conversion,
// 16-tap FIR and 256-point FFT into channels, with an optional fused epilogue that applies the
// sub-sample delay phase and bandpass (Sections 3, 4.3) and writes the corner-turned layout.
//
// One CTA filters up to 64 consecutive spectra of one (station, subband) stream, both
// polarisations.  Thread p owns FIR point p: it slides a 16-frame window of dual-pol samples
// through registers (one coalesced 8-byte load per frame per thread, each frame read once per CTA)
// and produces v_m[p] for 16 spectra into shared memory.  The 32 FFTs of a tile (16 spectra x 2
// pols) then run as 16x16 decompositions, 16 threads per transform: a 16-point DFT in registers,
// a twiddle from a shared table, a swizzled in-place shared-memory transpose, and a second
// 16-point DFT.
#include <cuda_fp16.h>

#include "lbf_internal.cuh"

namespace lbf {
namespace {

constexpr int kThreads = 256;
constexpr int kTile = 16;        // spectra per shared-memory tile
constexpr int kTilesPerCta = 4;  // spectra per CTA = 64
constexpr int kSpectraPerCta = kTile * kTilesPerCta;

template <int BITS> struct SampleIO;
template <> struct SampleIO<16> {   // X.re, X.im, Y.re, Y.im as four little-endian int16
  using word = uint2;
  __device__ static float4 cvt(uint2 u) {
    return make_float4((float)(int16_t)(u.x & 0xffffu), (float)(int16_t)(u.x >> 16),
                       (float)(int16_t)(u.y & 0xffffu), (float)(int16_t)(u.y >> 16));
  }
};
template <> struct SampleIO<8> {    // X.re, X.im, Y.re, Y.im as four int8
  using word = uint32_t;
  __device__ static float4 cvt(uint32_t u) {
    return make_float4((float)(int8_t)(u & 0xffu), (float)(int8_t)((u >> 8) & 0xffu),
                       (float)(int8_t)((u >> 16) & 0xffu), (float)(int8_t)(u >> 24));
  }
};

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// In-place 4-point DFT, y_k = sum_n x_n exp(-2 pi i n k / 4).
__device__ __forceinline__ void dft4(float2 &x0, float2 &x1, float2 &x2, float2 &x3) {
  const float2 a = f2add(x0, x2), b = f2sub(x0, x2), c = f2add(x1, x3), d = f2sub(x1, x3);
  x0 = f2add(a, c);
  x2 = f2sub(a, c);
  x1 = make_float2(b.x + d.y, b.y - d.x);   // b - i d
  x3 = make_float2(b.x - d.y, b.y + d.x);   // b + i d
}

// exp(-2 pi i j / 16) for the j = n2 * k1 products that occur in a 4x4 split.
__device__ __forceinline__ float2 w16(int j) {
  constexpr float c1 = 0.92387953251128674f, s1 = 0.38268343236508977f, r2 = 0.70710678118654752f;
  switch (j) {
    case 1: return make_float2(c1, -s1);
    case 2: return make_float2(r2, -r2);
    case 3: return make_float2(s1, -c1);
    case 4: return make_float2(0.f, -1.f);
    case 6: return make_float2(-r2, -r2);
    case 9: return make_float2(-c1, s1);
    default: return make_float2(1.f, 0.f);
  }
}

// 16-point DFT A[k] = sum_n a[n] exp(-2 pi i n k / 16), natural order in and out (n = 4 n1 + n2,
// k = k1 + 4 k2: four 4-point DFTs over n1, twiddles, four 4-point DFTs over n2).
__device__ __forceinline__ void dft16(float2 (&a)[16]) {
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4(a[n2], a[4 + n2], a[8 + n2], a[12 + n2]);
#pragma unroll
  for (int n2 = 1; n2 < 4; ++n2)
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1) a[4 * k1 + n2] = cmul(a[4 * k1 + n2], w16(n2 * k1));
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4(a[4 * k1], a[4 * k1 + 1], a[4 * k1 + 2], a[4 * k1 + 3]);
  float2 t[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) t[r] = a[4 * (r & 3) + (r >> 2)];
#pragma unroll
  for (int r = 0; r < 16; ++r) a[r] = t[r];
}

struct PpfSmem {
  float2 v[kP][kTile][kN];   // FIR outputs, then FFT scratch, then corner-turn staging
  float2 tw[kN];             // exp(-2 pi i n / 256)
  float2 gain[kN];           // bandpass * delay phasor per channel (fused epilogue)
};

// Output modes: the channelised layout, the FP32 corner-turned layout, or the FP16 corner-turned
// layout of the tensor-core beam former ([F][N][P][M][Kpad] with station s at k = 2s (re), 2s+1
// (im); a hi plane fp16(Y) and optionally a lo plane fp16(Y - hi)).
enum PpfMode { MODE_CHAN = 0, MODE_CT32 = 1, MODE_CT16 = 2 };

struct PpfOut {
  float2 *f32;
  __half *hi, *lo;
  int kpad;
};

template <int BITS, int MODE>
__global__ void __launch_bounds__(kThreads, 2)
ppf_kernel(Geometry g, const typename SampleIO<BITS>::word *__restrict__ in,
           const typename SampleIO<BITS>::word *__restrict__ hist, PpfOut po, int chunks) {
  using word = typename SampleIO<BITS>::word;
  constexpr bool CT = MODE != MODE_CHAN;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PpfSmem &sm = *reinterpret_cast<PpfSmem *>(smem_raw);
  float2 *__restrict__ out = po.f32;

  const int tid = threadIdx.x;
  int s, f, chunk;
  if (MODE == MODE_CT16) {   // stations fastest: the scattered 4-byte station slots of one
    s = (int)(blockIdx.x % g.S);                 // (channel, pol, spectrum) row are written by
    const long long rest = blockIdx.x / g.S;     // neighbouring CTAs and merge in L2
    chunk = (int)(rest % chunks);
    f = (int)(rest / chunks);
  } else {
    const long long sf = blockIdx.x / chunks;    // stream index s * F + f
    chunk = (int)(blockIdx.x - sf * chunks);
    s = (int)(sf / g.F);
    f = (int)(sf - (long long)s * g.F);
  }
  const long long sf = (long long)s * g.F + f;
  const int m0 = chunk * kSpectraPerCta;
  const int m_end = min(g.M, m0 + kSpectraPerCta);

  sm.tw[tid] = g.twiddle[tid];
  if (CT) {
    // Y = X * bp[c] * exp(+2 pi i (f0 tau_s + df_c (tau_s - n_s Ts))), phase in FP64 cycles
    const int c = tid;
    const double df = (double)(c - kN / 2) * (g.fs / kN);
    const double phi = g.f0[f] * g.tau[s] + df * g.resid[s];
    const float2 ph = unit_phasor_cycles(phi);
    const float b = g.bandpass[c];
    sm.gain[c] = make_float2(b * ph.x, b * ph.y);
  }

  // x'[j] = x[j - d_s]; block-relative x' index j lives at extended index H - d_s + j of
  // [history (H samples) | block (T samples)].
  const int p = tid;
  const long long base = (long long)g.H - g.dshift[s] + p;
  const word *hs = hist + sf * g.H;
  const word *bs = in + sf * g.T;
  auto load_frame = [&](int r) -> float4 {   // sample x'[r N + p], frame r >= -15, r < M
    const long long e = base + (long long)r * kN;
    const word w = (e < g.H) ? hs[e] : bs[e - g.H];
    return SampleIO<BITS>::cvt(w);
  };

  float h[kL];
#pragma unroll
  for (int t = 0; t < kL; ++t) h[t] = g.taps[t * kN + p];

  float4 win[kL];   // frame r is kept in slot r & 15
#pragma unroll
  for (int i = 0; i < kL - 1; ++i) win[i + 1] = load_frame(m0 - (kL - 1) + i);

  const int j = tid & 15;     // lane within a 16-thread transform group
  const int grp = tid >> 4;   // transform group: spectrum q of the tile

  for (int mt = m0; mt < m_end; mt += kTile) {
    // ---- FIR: v_m[p] = sum_t h[tN + p] x'[(m - 15 + t) N + p], for 16 spectra
#pragma unroll
    for (int q = 0; q < kTile; ++q) {
      const int m = mt + q;
      win[q] = (m < m_end) ? load_frame(m) : make_float4(0.f, 0.f, 0.f, 0.f);
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int t = 0; t < kL; ++t) {
        const float4 x = win[(q + 1 + t) & 15];
        acc.x = fmaf(h[t], x.x, acc.x);
        acc.y = fmaf(h[t], x.y, acc.y);
        acc.z = fmaf(h[t], x.z, acc.z);
        acc.w = fmaf(h[t], x.w, acc.w);
      }
      sm.v[0][q][p] = make_float2(acc.x, acc.y);
      sm.v[1][q][p] = make_float2(acc.z, acc.w);
    }
    __syncthreads();

    // ---- FFT-256 of the 32 transforms (pol = round, spectrum q = group), 16 threads each
#pragma unroll 1
    for (int pol = 0; pol < kP; ++pol) {
      float2 *row = sm.v[pol][grp];
      float2 a[16];
#pragma unroll
      for (int p1 = 0; p1 < 16; ++p1) a[p1] = row[16 * p1 + j];   // thread j = p2
      __syncwarp();
      dft16(a);
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) row[k1 * 16 + (j ^ k1)] = cmul(a[k1], sm.tw[j * k1]);
      __syncwarp();
#pragma unroll
      for (int p2 = 0; p2 < 16; ++p2) a[p2] = row[j * 16 + (p2 ^ j)];   // thread j = k1
      dft16(a);   // a[k2] = X[j + 16 k2]
      const int m = mt + grp;
      if (MODE == MODE_CT16) {
        if (m < m_end) {
          const long long rowbase = (((long long)f * kN) * kP + pol) * g.M + m;
#pragma unroll
          for (int k2 = 0; k2 < 16; ++k2) {
            const int c = j + 16 * ((k2 + 8) & 15);
            const float2 v = cmul(a[k2], sm.gain[c]);
            const long long idx = (rowbase + (long long)c * kP * g.M) * po.kpad + 2 * s;
            const __half2 hi = __floats2half2_rn(v.x, v.y);
            *reinterpret_cast<__half2 *>(po.hi + idx) = hi;
            if (po.lo)
              *reinterpret_cast<__half2 *>(po.lo + idx) =
                  __floats2half2_rn(v.x - __low2float(hi), v.y - __high2float(hi));
          }
        }
      } else if (!CT) {
        if (m < m_end) {
          float2 *dst = out + ((((long long)f * g.S + s) * kP + pol) * g.M + m) * kN;
#pragma unroll
          for (int k2 = 0; k2 < 16; ++k2) dst[j + 16 * ((k2 + 8) & 15)] = a[k2];   // c = (k + N/2) mod N
        }
      } else {
        __syncthreads();   // every group has read its row: the pol plane becomes staging [c][q]
        float2 *stage = &sm.v[pol][0][0];
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) {
          const int c = j + 16 * ((k2 + 8) & 15);
          stage[c * 16 + (grp ^ (c & 15))] = cmul(a[k2], sm.gain[c]);
        }
        __syncthreads();
        // ct[f][c][s][pol][m]: runs of 16 consecutive spectra per (c, pol)
        const int q = tid & 15;
        if (mt + q < m_end) {
#pragma unroll 4
          for (int pass = 0; pass < kN / 16; ++pass) {
            const int c = pass * 16 + (tid >> 4);
            out[((((long long)f * kN + c) * g.S + s) * kP + pol) * g.M + mt + q] =
                stage[c * 16 + (q ^ (c & 15))];
          }
        }
      }
    }
    __syncthreads();
  }
}

template <int BITS>
__global__ void hist_update_kernel(long long total, int H, int T,
                                   const typename SampleIO<BITS>::word *__restrict__ in,
                                   const typename SampleIO<BITS>::word *__restrict__ hist,
                                   typename SampleIO<BITS>::word *__restrict__ nhist) {
  // new history = samples T .. T+H-1 of [history | block]
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long sf = i / H;
    const int e = (int)(i - sf * H);
    const long long src = (long long)T + e;
    nhist[i] = (src < H) ? hist[sf * H + src] : in[sf * T + (src - H)];
  }
}

template <int BITS, int MODE>
cudaError_t launch_ppf_t(const Geometry &g, const void *in, const void *hist, PpfOut po, cudaStream_t st) {
  using word = typename SampleIO<BITS>::word;
  const int chunks = (g.M + kSpectraPerCta - 1) / kSpectraPerCta;
  const long long ctas = (long long)g.S * g.F * chunks;
  if (ctas == 0) return cudaSuccess;
  const size_t smem = sizeof(PpfSmem);
  auto kern = ppf_kernel<BITS, MODE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)ctas, kThreads, smem, st>>>(g, (const word *)in, (const word *)hist, po, chunks);
  return cudaGetLastError();
}

template <int BITS>
cudaError_t launch_ppf_bits(const Geometry &g, const void *in, const void *hist, float2 *chan, float2 *ct,
                            const Ct16Out *ct16, cudaStream_t st) {
  PpfOut po{nullptr, nullptr, nullptr, 0};
  if (ct16) {
    po.hi = reinterpret_cast<__half *>(ct16->hi);
    po.lo = reinterpret_cast<__half *>(ct16->lo);
    po.kpad = ct16->kpad;
    return launch_ppf_t<BITS, MODE_CT16>(g, in, hist, po, st);
  }
  if (ct) {
    po.f32 = ct;
    return launch_ppf_t<BITS, MODE_CT32>(g, in, hist, po, st);
  }
  po.f32 = chan;
  return launch_ppf_t<BITS, MODE_CHAN>(g, in, hist, po, st);
}

}  // namespace

cudaError_t launch_ppf(const Geometry &g, int bits, const void *in, const void *hist, float2 *chan,
                       float2 *ct, cudaStream_t st, const Ct16Out *ct16) {
  return bits == 16 ? launch_ppf_bits<16>(g, in, hist, chan, ct, ct16, st)
                    : launch_ppf_bits<8>(g, in, hist, chan, ct, ct16, st);
}

cudaError_t launch_hist_update(const Geometry &g, int bits, const void *in, const void *hist,
                               void *new_hist, cudaStream_t st) {
  const long long total = (long long)g.S * g.F * g.H;
  if (total == 0) return cudaSuccess;
  const int threads = 256;
  const long long want = (total + threads - 1) / threads;
  const unsigned blocks = (unsigned)(want < 152LL * 16 ? want : 152LL * 16);
  if (bits == 16)
    hist_update_kernel<16><<<blocks, threads, 0, st>>>(total, g.H, g.T, (const uint2 *)in,
                                                       (const uint2 *)hist, (uint2 *)new_hist);
  else
    hist_update_kernel<8><<<blocks, threads, 0, st>>>(total, g.H, g.T, (const uint32_t *)in,
                                                      (const uint32_t *)hist, (uint32_t *)new_hist);
  return cudaGetLastError();
}

}  // namespace lbf
