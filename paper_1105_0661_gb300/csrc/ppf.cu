// Poly-phase filter bank of Section 4.2: integer sample shift (Section 3), int->float conversion,
// 16-tap FIR and 256-point FFT into channels, with an optional fused epilogue that applies the
// sub-sample delay phase and bandpass (Sections 3, 4.3) and writes a corner-turned layout.
//
// One CTA filters one polarisation of up to 128 consecutive spectra of one (station, subband)
// stream in tiles of 16 spectra, with 256 threads: thread p owns FIR point p.  Two CTAs fit on an
// SM, so one CTA's FIR (FP32-pipe bound) overlaps the other's FFT (shared-memory latency bound);
// the two polarisations of a stream chunk are neighbouring CTAs, and the second reads the dual-pol
// input from L2.
//  * The tile's input samples arrive through a two-stage cp.async ring in shared memory (whole
//    dual-pol samples, issued one tile ahead), so global-load latency overlaps the filtering and
//    the FFTs of the tile before.
//  * Each thread converts its polarisation exactly to float with the 2^23 magic-number method
//    (integer ops + one packed add instead of the conversion pipe) and slides a 16-frame window
//    of complex values through registers, producing v_m[p] for 16 spectra into shared memory.
// The 16 FFTs of a tile then run as 16x16 decompositions, 16 threads per transform: a 16-point DFT
// in registers (packed FP32x2 butterflies), a twiddle from a shared table, an in-place transpose
// through padded shared-memory rows, and a second 16-point DFT.
#include <cuda_fp16.h>

#include <type_traits>

#include "fft16.cuh"
#include "lbf_internal.cuh"

namespace lbf {
namespace {

constexpr int kThreads = 256;
constexpr int kTile = 16;                  // spectra per tile: 16 transforms = one FFT round
// Spectra per CTA: as many as still give at least kMinCtas CTAs (16 waves of two CTAs per SM on
// 152 SMs), since each CTA's setup (taps, FIR window, delay phasors) is then spread over more
// tiles: the whole 768-spectrum block of a stream for the LOFAR observation (4.7 % faster than 128
// spectra per CTA), 16 spectra for an observation of a few streams.
constexpr long long kMinCtas = 152LL * 2 * 16;
constexpr int kStages = 2;                 // input ring depth (tiles)
constexpr float kMagic16 = 8421376.0f;     // 2^23 + 2^15
constexpr float kMagic8 = 8388736.0f;      // 2^23 + 2^7

template <int BITS> struct SampleIO;
template <> struct SampleIO<16> {   // X.re, X.im, Y.re, Y.im as four little-endian int16
  using word = uint2;
  // One polarisation (re, im as two int16 in a 32-bit word) to float: the bits
  // 0x4B00 | (v + 2^15) are the float 2^23 + v + 2^15, so one packed subtract is exact.
  __device__ static float2 cvt_pol(const word &w, int pol) {
    const uint32_t a = (pol ? w.y : w.x) ^ 0x80008000u;
    return __fadd2_rn(make_float2(__uint_as_float(__byte_perm(a, 0x4B00u, 0x5410u)),
                                  __uint_as_float(__byte_perm(a, 0x4B00u, 0x5432u))),
                      make_float2(-kMagic16, -kMagic16));
  }
};
template <> struct SampleIO<8> {    // X.re, X.im, Y.re, Y.im as four int8
  using word = uint32_t;
  // One polarisation (two int8) to float: 0x4B0000 | (v + 2^7) is the float 2^23 + v + 2^7.
  __device__ static float2 cvt_pol(const word &w, int pol) {
    const uint32_t a = (w ^ 0x80808080u) >> (16 * pol);
    return __fadd2_rn(make_float2(__uint_as_float(__byte_perm(a, 0x4B00u, 0x5440u)),
                                  __uint_as_float(__byte_perm(a, 0x4B00u, 0x5441u))),
                      make_float2(-kMagic8, -kMagic8));
  }
};

// A transform's 256 points are kept as 16 rows of 16 with one float2 of padding per row, so that
// both the row and the column walks of the 16 x 16 decomposition are conflict-free with fixed
// per-thread offsets (no index arithmetic in the FFT).
constexpr int kRow = 16 * 17;
template <int BITS>
struct PpfSmem {
  using word = typename SampleIO<BITS>::word;
  static constexpr int kAlign = 16 / (int)sizeof(word);     // samples per 16 bytes
  static constexpr int kSlot = kTile * kN + kAlign;         // one tile of frames + alignment slack
  float2 v[kTile][kRow];                                    // 34 KB: FIR out -> FFT -> staging
  word in[kStages][kSlot];                                  // input ring (64 KB int16, 32 KB int8)
  float2 tw[kN];                                            // [k1][j] = exp(-2 pi i j k1 / 256)
  float2 gain[kN];                                          // bandpass * delay phasor per channel
};

// Output modes: the channelised layout, the FP32 corner-turned layout, or the FP16 layout of the
// tensor-core beam former ([F*N][M/32][Kpad][P][32] with station s in rows k = 2s (re), 2s+1 (im);
// a hi plane fp16(Y) and optionally a lo plane fp16(Y - hi)).
enum PpfMode { MODE_CHAN = 0, MODE_CT32 = 1, MODE_CT16 = 2 };

struct PpfOut {
  float2 *f32;
  __half *hi, *lo;
  int kpad;
};

__device__ __forceinline__ void cp_async(void *smem_dst, const void *gmem_src, int bytes) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
  if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gmem_src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// One work item: polarisation pol of spectra [chunk * spc, (chunk + 1) * spc) of stream (s, f),
// spc a multiple of 16.
template <int BITS, int MODE>
__device__ __forceinline__ void ppf_item(const Geometry &g, const typename SampleIO<BITS>::word *__restrict__ in,
                                         const typename SampleIO<BITS>::word *__restrict__ hist, const PpfOut &po,
                                         int s, int f, int pol, int chunk, int spc, unsigned char *smem_raw) {
  using word = typename SampleIO<BITS>::word;
  constexpr bool CT = MODE != MODE_CHAN;
  PpfSmem<BITS> &sm = *reinterpret_cast<PpfSmem<BITS> *>(smem_raw);
  float2 *__restrict__ out = po.f32;

  const int tid = threadIdx.x;
  const long long sf = (long long)s * g.F + f;
  const int m0 = chunk * spc;
  const int m_end = min(g.M, m0 + spc);
  const int ntiles = (m_end - m0 + kTile - 1) / kTile;
  constexpr int kAlign = PpfSmem<BITS>::kAlign;

  sm.tw[tid] = g.twiddle[(tid & 15) * (tid >> 4)];
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
  // [history (H samples) | block (T samples)].  Frames r >= -15, r < M.
  const int p = tid;               // this thread's FIR point
  const int dsh = g.dshift[s];
  const long long base = (long long)g.H - dsh + p;
  const word *hs = hist + sf * g.H;
  const word *bs = in + sf * g.T;
  auto src_of = [&](int r) -> const word * {
    const long long e = base + (long long)r * kN;
    return (e < g.H) ? hs + e : bs + (e - g.H);
  };
  // Tile t's frames start at block sample e0 = mt N - d_s.  A tile wholly inside the block (e0 >= 0)
  // is one contiguous run of samples: it is copied as 16-byte pieces of the aligned run that covers
  // it (never past the stream's end, T being a multiple of N), and its frames start at slot offset
  // e0 mod kAlign.  A tile that reaches into the history takes one copy per sample.
  const bool in16 = ((reinterpret_cast<uintptr_t>(in) & 15) == 0);
  auto slot_off = [&](int mt) -> int {
    const long long e0 = (long long)mt * kN - dsh;
    return (in16 && e0 >= 0) ? (int)(e0 & (kAlign - 1)) : 0;
  };
  auto issue_tile = [&](int t) {
    if (t < ntiles) {
      const int mt = m0 + t * kTile;
      const int nfr = min(kTile, m_end - mt);
      word *slot = sm.in[t % kStages];
      const long long e0 = (long long)mt * kN - dsh;
      if (in16 && e0 >= 0) {
        const long long a = e0 & ~(long long)(kAlign - 1);
        const int nchunks = (int)((e0 - a + (long long)nfr * kN + kAlign - 1) / kAlign);
        const char *src = reinterpret_cast<const char *>(bs + a);
        char *dst = reinterpret_cast<char *>(slot);
        // nchunks is kTile N / kAlign + (0 or 1) for full tiles: whole rounds at fixed offsets
        const char *s0 = src + 16 * tid;
        char *d0 = dst + 16 * tid;
        const int rounds = nchunks / kThreads;
        if (rounds == kTile * kN / kAlign / kThreads) {
#pragma unroll
          for (int r = 0; r < kTile * kN / kAlign / kThreads; ++r) cp_async16(d0 + 16 * kThreads * r, s0 + 16 * kThreads * r);
        } else {
          for (int r = 0; r < rounds; ++r) cp_async16(d0 + 16 * kThreads * r, s0 + 16 * kThreads * r);
        }
        const int i = rounds * kThreads + tid;
        if (i < nchunks) cp_async16(dst + 16 * i, src + 16 * i);
      } else {
#pragma unroll
        for (int q = 0; q < kTile; ++q)
          if (q < nfr) cp_async(slot + q * kN + p, src_of(mt + q), (int)sizeof(word));
      }
    }
    cp_async_commit();
  };
  issue_tile(0);

  float2 h2[kL];   // (h, h): one packed FMA updates both components
#pragma unroll
  for (int t = 0; t < kL; ++t) { const float hv = g.taps[t * kN + p]; h2[t] = make_float2(hv, hv); }

  float2 win[kL];   // frame r of this pol is kept in slot r & 15 (m0 is a multiple of 16)
#pragma unroll
  for (int i = 0; i < kL - 1; ++i) win[i + 1] = SampleIO<BITS>::cvt_pol(*src_of(m0 - (kL - 1) + i), pol);

  const int j = tid & 15;          // lane within a 16-thread transform group
  const int gq = tid >> 4;         // the group's spectrum within the tile
  const int pv = 17 * (p >> 4) + (p & 15);   // point p in a padded row

  for (int t = 0; t < ntiles; ++t) {
    const int mt = m0 + t * kTile;
    issue_tile(t + 1);
    cp_async_wait<1>();            // this thread's copies of tile t have landed
    __syncthreads();               // ... and everyone's
    // ---- FIR: v_m[p] = sum_t h[tN + p] x'[(m - 15 + t) N + p], 16 spectra, this pol
    const word *fr = sm.in[t % kStages] + slot_off(mt) + p;
    float2 *vout = &sm.v[0][pv];
    auto fir = [&](auto full) {
#pragma unroll
      for (int q = 0; q < kTile; ++q) {
        if (decltype(full)::value || mt + q < m_end) win[q] = SampleIO<BITS>::cvt_pol(fr[q * kN], pol);
        else win[q] = make_float2(0.f, 0.f);
        // two partial sums per component halve the FMA dependency chain
        float2 acc = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
#pragma unroll
        for (int tap = 0; tap < kL; tap += 2) {
          acc = __ffma2_rn(h2[tap], win[(q + 1 + tap) & 15], acc);
          acc1 = __ffma2_rn(h2[tap + 1], win[(q + 2 + tap) & 15], acc1);
        }
        vout[q * kRow] = __fadd2_rn(acc, acc1);
      }
    };
    if (mt + kTile <= m_end) fir(std::true_type());
    else fir(std::false_type());
    __syncthreads();

    // ---- FFT-256 of the 16 transforms (spectra) of the tile, 16 threads each:
    // n = 16 p1 + p2, k = k1 + 16 k2; thread j first owns column p2 = j, then row k1 = j
    float2 *row = sm.v[gq];
    float2 a[16];
#pragma unroll
    for (int p1 = 0; p1 < 16; ++p1) a[p1] = row[17 * p1 + j];
    dft16(a);
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) row[17 * k1 + j] = cmul(a[k1], sm.tw[16 * k1 + j]);
    __syncwarp();
#pragma unroll
    for (int p2 = 0; p2 < 16; ++p2) a[p2] = row[17 * j + p2];
    dft16(a);   // a[k2] = X[j + 16 k2]
    const int m = mt + gq;
    if (MODE == MODE_CT16) {
      __syncthreads();   // every group has read its row: the buffer becomes staging [c][q]
      float2 *stage = &sm.v[0][0];
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) {
        const int c = j + 16 * ((k2 + 8) & 15);
        stage[c * kTile + (gq ^ (c & 15))] = cmul(a[k2], sm.gain[c]);
      }
      __syncthreads();
      // [F*N][Mt][Kpad][P][32]: rows k = 2s (re) and 2s+1 (im).  Thread (channel c, h8) packs
      // 8 consecutive spectra into one 16-byte store per plane and component; spectra at or past
      // the block's end go out as zeros (the pad columns of the last tile).
      const int mb = tc_tiles(g.M);
      const bool full = mt + kTile <= m_end;
      const int h8 = tid & 1;
      const int m0 = mt + 8 * h8;
#pragma unroll
      for (int pass = 0; pass < kN / (kThreads / 2); ++pass) {
        const int c = pass * (kThreads / 2) + (tid >> 1);
        const float2 *srow = stage + c * kTile;
        uint32_t hr[4], hm[4], lr[4], lm[4];
#pragma unroll
        for (int k = 0; k < 8; k += 2) {
          float2 v0 = srow[(8 * h8 + k) ^ (c & 15)], v1 = srow[(8 * h8 + k + 1) ^ (c & 15)];
          if (!full) {
            if (m0 + k >= m_end) v0 = make_float2(0.f, 0.f);
            if (m0 + k + 1 >= m_end) v1 = make_float2(0.f, 0.f);
          }
          const __half2 h_re = __floats2half2_rn(v0.x, v1.x), h_im = __floats2half2_rn(v0.y, v1.y);
          const float2 f_re = __half22float2(h_re), f_im = __half22float2(h_im);
          const __half2 l_re = __floats2half2_rn(v0.x - f_re.x, v1.x - f_re.y);
          const __half2 l_im = __floats2half2_rn(v0.y - f_im.x, v1.y - f_im.y);
          hr[k / 2] = *reinterpret_cast<const uint32_t *>(&h_re);
          hm[k / 2] = *reinterpret_cast<const uint32_t *>(&h_im);
          lr[k / 2] = *reinterpret_cast<const uint32_t *>(&l_re);
          lm[k / 2] = *reinterpret_cast<const uint32_t *>(&l_im);
        }
        const long long re = ((((long long)f * kN + c) * mb + (m0 >> 5)) * po.kpad + 2 * s) * 64 + pol * 32 + (m0 & 31);
        *reinterpret_cast<uint4 *>(po.hi + re) = make_uint4(hr[0], hr[1], hr[2], hr[3]);
        *reinterpret_cast<uint4 *>(po.hi + re + 64) = make_uint4(hm[0], hm[1], hm[2], hm[3]);
        if (po.lo) {
          *reinterpret_cast<uint4 *>(po.lo + re) = make_uint4(lr[0], lr[1], lr[2], lr[3]);
          *reinterpret_cast<uint4 *>(po.lo + re + 64) = make_uint4(lm[0], lm[1], lm[2], lm[3]);
        }
      }
    } else if (!CT) {
      if (m < m_end) {
        float2 *dst = out + ((((long long)f * g.S + s) * kP + pol) * g.M + m) * kN;
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) dst[j + 16 * ((k2 + 8) & 15)] = a[k2];   // c = (k + N/2) mod N
      }
    } else {
      __syncthreads();   // every group has read its row: the buffer becomes staging [c][q]
      float2 *stage = &sm.v[0][0];
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) {
        const int c = j + 16 * ((k2 + 8) & 15);
        stage[c * kTile + (gq ^ (c & 15))] = cmul(a[k2], sm.gain[c]);
      }
      __syncthreads();
      // ct[f][c][s][pol][m]: runs of 16 consecutive spectra (128 B) per channel.  Eight threads
      // write a run, two spectra each as one 16-byte store (rows 16-byte aligned when M is even),
      // so a warp's store covers four whole 128-byte runs.  Pass k writes channels 32 k + tid / 8.
      const int pr = tid & 7;
      const int m0 = mt + 2 * pr;
      const bool vec = (g.M & 1) == 0 && m0 + 1 < m_end;
      const int c0 = tid >> 3;
      const float2 *srow = stage + c0 * kTile;
      const int sw = c0 & 15;   // the swizzle of every channel this thread writes
      float2 *dst = out + ((((long long)f * kN + c0) * g.S + s) * kP + pol) * g.M + m0;
      const long long cstep = (long long)(kThreads / 8) * g.S * kP * g.M;
#pragma unroll
      for (int pass = 0; pass < kN / (kThreads / 8); ++pass, dst += cstep) {
        const float2 v0 = srow[pass * (kThreads / 8) * kTile + ((2 * pr) ^ sw)];
        const float2 v1 = srow[pass * (kThreads / 8) * kTile + ((2 * pr + 1) ^ sw)];
        if (vec) {
          *reinterpret_cast<float4 *>(dst) = make_float4(v0.x, v0.y, v1.x, v1.y);
        } else {
          if (m0 < m_end) dst[0] = v0;
          if (m0 + 1 < m_end) dst[1] = v1;
        }
      }
    }
    __syncthreads();
  }
  cp_async_wait<0>();
}

// Polarisation fastest in the CTA index: the two CTAs of a stream chunk read the same input run.
template <int BITS, int MODE>
__global__ void __launch_bounds__(kThreads, 2)
ppf_kernel(Geometry g, const typename SampleIO<BITS>::word *__restrict__ in,
           const typename SampleIO<BITS>::word *__restrict__ hist, PpfOut po, int chunks, int spc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int s, f, chunk;
  const int pol = (int)(blockIdx.x & 1);
  const long long item = blockIdx.x >> 1;
  if (MODE == MODE_CT16) {   // then stations: neighbouring CTAs fill neighbouring K rows of
    s = (int)(item % g.S);                       // the same (channel) planes
    const long long rest = item / g.S;
    chunk = (int)(rest % chunks);
    f = (int)(rest / chunks);
  } else {
    const long long sf = item / chunks;          // stream index s * F + f
    chunk = (int)(item - sf * chunks);
    s = (int)(sf / g.F);
    f = (int)(sf - (long long)s * g.F);
  }
  ppf_item<BITS, MODE>(g, in, hist, po, s, f, pol, chunk, spc, smem_raw);
}

// Persistent filter bank over the blocks of several observations (a batch): CTAs take work items
// (stream, spectrum chunk, polarisation) from a shared counter until all groups are done.
__global__ void __launch_bounds__(kThreads, 2)
ppf_group_kernel(const PpfGroup *__restrict__ grp, int ngrp, long long total, unsigned long long *counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long item_s;
  for (;;) {
    if (threadIdx.x == 0) item_s = (long long)atomicAdd(counter, 1ull);
    __syncthreads();
    const long long item = item_s;
    __syncthreads();
    if (item >= total) break;
    int o = 0;
    while (o + 1 < ngrp && grp[o + 1].first_item <= item) ++o;
    const PpfGroup &G = grp[o];
    const long long local = (item - G.first_item) >> 1;
    const int pol = (int)((item - G.first_item) & 1);
    const long long sf = local / G.chunks;
    const int chunk = (int)(local - sf * G.chunks);
    const int s = (int)(sf / G.g.F), f = (int)(sf - (long long)s * G.g.F);
    if (G.tc) {   // tensor-core plan: FP16 hi+lo planes
      PpfOut po{nullptr, reinterpret_cast<__half *>(G.ct16.hi), reinterpret_cast<__half *>(G.ct16.lo), G.ct16.kpad};
      if (G.bits == 16)
        ppf_item<16, MODE_CT16>(G.g, (const uint2 *)G.in, (const uint2 *)G.hist, po, s, f, pol, chunk, G.spc, smem_raw);
      else
        ppf_item<8, MODE_CT16>(G.g, (const uint32_t *)G.in, (const uint32_t *)G.hist, po, s, f, pol, chunk, G.spc, smem_raw);
    } else {
      PpfOut po{G.ct, nullptr, nullptr, 0};
      if (G.bits == 16)
        ppf_item<16, MODE_CT32>(G.g, (const uint2 *)G.in, (const uint2 *)G.hist, po, s, f, pol, chunk, G.spc, smem_raw);
      else
        ppf_item<8, MODE_CT32>(G.g, (const uint32_t *)G.in, (const uint32_t *)G.hist, po, s, f, pol, chunk, G.spc, smem_raw);
    }
  }
}

// History update of every observation of a batch: element i of the concatenated histories.
__global__ void hist_group_kernel(const PpfGroup *__restrict__ grp, int ngrp, long long total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int o = 0;
    while (o + 1 < ngrp && grp[o + 1].first_hist <= i) ++o;
    const PpfGroup &G = grp[o];
    const long long j = i - G.first_hist;
    const long long sf = j / G.g.H;
    const int e = (int)(j - sf * G.g.H);
    const long long src = (long long)G.g.T + e;
    if (G.bits == 16) {
      const uint2 *in = (const uint2 *)G.in, *h = (const uint2 *)G.hist;
      ((uint2 *)G.new_hist)[j] = (src < G.g.H) ? h[sf * G.g.H + src] : in[sf * G.g.T + (src - G.g.H)];
    } else {
      const uint32_t *in = (const uint32_t *)G.in, *h = (const uint32_t *)G.hist;
      ((uint32_t *)G.new_hist)[j] = (src < G.g.H) ? h[sf * G.g.H + src] : in[sf * G.g.T + (src - G.g.H)];
    }
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
  const long long streams = (long long)g.S * g.F * kP;
  if (streams == 0 || g.M == 0) return cudaSuccess;
  const long long want = (kMinCtas + streams - 1) / streams;      // chunks per stream wanted
  const int spc = (int)((((long long)g.M + want - 1) / want + kTile - 1) / kTile) * kTile;
  const int chunks = (g.M + spc - 1) / spc;
  const long long ctas = streams * chunks;
  if (ctas == 0) return cudaSuccess;
  const size_t smem = sizeof(PpfSmem<BITS>);
  auto kern = ppf_kernel<BITS, MODE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)ctas, kThreads, smem, st>>>(g, (const word *)in, (const word *)hist, po, chunks, spc);
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

cudaError_t launch_ppf_group(const PpfGroup *d_groups, int ngrp, long long total, unsigned long long *counter,
                             int ctas, cudaStream_t st) {
  if (total == 0) return cudaSuccess;
  const size_t smem = sizeof(PpfSmem<16>);
  cudaError_t e = cudaFuncSetAttribute(ppf_group_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  ppf_group_kernel<<<ctas, kThreads, smem, st>>>(d_groups, ngrp, total, counter);
  return cudaGetLastError();
}

cudaError_t launch_hist_group(const PpfGroup *d_groups, int ngrp, long long total, cudaStream_t st) {
  if (total == 0) return cudaSuccess;
  const long long want = (total + 255) / 256;
  hist_group_kernel<<<(unsigned)(want < 152LL * 16 ? want : 152LL * 16), 256, 0, st>>>(d_groups, ngrp, total);
  return cudaGetLastError();
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
