// Poly-phase filter bank of Section 4.2: integer sample shift (Section 3), int->float conversion,
// 16-tap FIR and 256-point FFT into channels, with an optional fused epilogue that writes a
// corner-turned layout: in FP32 with the sub-sample delay phase and bandpass applied (Sections 3,
// 4.3), or as the FP16 planes of the tensor-core beam former, whose weights carry that phase and
// the bandpass instead (the phase has the weight phase's form; tables.cu folds it in).
//
// One 512-thread CTA filters both polarisations of up to `spc` consecutive spectra of one
// (station, subband) stream, in tiles of 16 spectra.  Each half of the CTA (256 threads) owns one
// polarisation; thread p of a half owns FIR point p.  The halves share the input staging and the
// per-channel tables and otherwise run on their own named barriers, so one half's FIR (FP32 pipe)
// overlaps the other half's FFT (shared memory).
//  * Input: a two-slot ring in shared memory filled by bulk asynchronous copies (cp.async.bulk,
//    completion counted on an mbarrier).  A tile inside the block is one contiguous run of
//    dual-polarisation samples: one copy of the 16-byte-aligned run that covers it (the integer
//    shift d_s only moves the start inside the slot).  The slot of tile t is refilled with tile
//    t + 2 by whichever half finishes reading it second.  A tile that reaches into the history
//    (the first one of a stream) is read from global memory directly.
//  * FIR: each thread converts its polarisation's samples exactly to float (on the conversion
//    pipe, which the FIR and FFT leave idle), slides a 16-frame window through registers and
//    sums 16 taps (each held as an (h, h) pair for packed FP32x2 FMAs), writing v_m[p] for the
//    tile's 16 spectra into the half's FIR buffer.
//  * FFT-256 as 16 x 16 (n = 16 p1 + p2, k = k1 + 16 k2).  Pass 1, in place: thread (m, p2) takes
//    column p2 of spectrum m, a 16-point DFT over p1 in registers and the twiddle
//    exp(-2 pi i p2 k1 / 256), and writes the results back over its own 16 points.  Pass 2:
//    thread (m = p & 15, k1 = p >> 4) reads 16 contiguous values, a 16-point DFT over p2 gives
//    X[k1 + 16 k2]; sixteen lanes then hold sixteen consecutive spectra of one channel (for the
//    FP32 output the delay phasor and bandpass are applied there).  The output is staged in the
//    tile's own (by then consumed) FIR buffer in the layout of a tensor-map box -- the FP32
//    corner turn as [256 channels][16 spectra] float2, the FP16 planes as [256 channels][the
//    station's two K rows][16 spectra] per plane -- and one thread per half writes it with tensor
//    stores that drain while the next tile is filtered: written from the lanes, the tile's 64 KB
//    left each SM in one burst at the end of the tile and stalled its warps (a runtime switch that
//    dropped the stores cut the pass-2 phase from 3.2-3.9k to 1.7-2.6k cycles per tile).  The
//    FP32 corner turn with odd M (no 16-byte strides for a tensor map) is written from the lanes
//    as whole 128-byte runs.
//  * Schedule over two tile buffers per half.  FP32 output: the whole FIR of tile t + 1 runs
//    inside pass 2 of tile t (pass 1 alone in the other phase), so that FMA-bound and
//    shared-memory-bound work are interleaved and the staged tile has a phase to drain before
//    that FIR refills its buffer (with lane stores the FIR is split 8/8 over the two passes).
//    FP16 planes: FIR, pass 1 and pass 2 in sequence; the stores of a tile must have read its
//    buffer before the FIR two tiles later refills it.
// Every wait on a copy is bounded: on expiry the CTA records DERR_PPF_INPUT in the device error
// word, stops, waits (bounded) for its copies in flight and returns.
#include <cuda.h>
#include <cuda_fp16.h>

#include <cstddef>
#include <cstring>
#include <type_traits>

#include "fft16.cuh"
#include "lbf_internal.cuh"

namespace lbf {
namespace {

constexpr int kHalf = 256;                 // threads per polarisation: thread p owns FIR point p
constexpr int kThreads = kP * kHalf;       // one CTA: both polarisations of a stream chunk
constexpr int kTile = 16;                  // spectra per tile: 16 transforms
// Spectra per CTA: as many as still give at least kMinCtas CTAs (16 waves of one CTA per SM on
// 152 SMs): the whole 768-spectrum block of a stream for the LOFAR observation, 16 spectra for an
// observation of a few streams.
constexpr long long kMinCtas = 152LL * 16;
constexpr int kStages = 2;                 // input ring depth (tiles)
constexpr int kRowV = 258;                 // float2 per transform row: 256 points + 2 of padding
constexpr uint32_t kWaitIters = 1u << 20;  // polls before a wait on a copy gives up
// FP32 corner turn with tensor stores: the FIR outputs of tile t + 1 computed during pass 1 of
// tile t (the rest during pass 2).  Rows [kFirA, 16) of a tile's buffer are refilled only in the
// pass-2 phase of the next tile, so they stage the channels [256 - kCtTma, 256) of the tile's
// output for the tensor store, from a 128-byte-aligned offset; the other channels are stored from
// the lanes.  Measured on the LOFAR block (FP32 filter bank 13.54 ms with every value stored from
// the lanes and 8 FIR outputs in each phase): kFirA = 8 (128 channels staged) 14.36 ms, 4 (192,
// spilling) 15.19 ms, 0 (all 256 staged, the whole FIR of the next tile inside pass 2) 13.14 ms.
constexpr int kFirA = 0;
constexpr int kCtStageOff = ((kFirA * kRowV * 8 + 127) / 128) * 128;                 // bytes
constexpr int kCtTma = (((kTile * kRowV * 8 - kCtStageOff) / 128) / 16) * 16 > kN
                           ? kN : (((kTile * kRowV * 8 - kCtStageOff) / 128) / 16) * 16;   // channels

template <int BITS> struct SampleIO;
template <> struct SampleIO<16> {   // X.re, X.im, Y.re, Y.im as four little-endian int16
  using word = uint2;
  static constexpr int kAlign = 2;   // samples per 16 bytes
  // polarisation pol's (re, im) of sample i as one 32-bit word
  __device__ static uint32_t pair(const word *base, long long i, int pol) {
    return reinterpret_cast<const uint32_t *>(base)[2 * i + pol];
  }
  // (re, im) int16 pair to float (exact): two conversions on the conversion pipe, leaving the FMA
  // pipe to the FIR and the FFT
  __device__ static float2 cvt(uint32_t a, int) {
    return make_float2((float)(int16_t)(a & 0xffffu), (float)(int16_t)(a >> 16));
  }
};
template <> struct SampleIO<8> {    // X.re, X.im, Y.re, Y.im as four int8
  using word = uint32_t;
  static constexpr int kAlign = 4;
  __device__ static uint32_t pair(const word *base, long long i, int) { return base[i]; }
  // polarisation pol's two int8 to float (exact)
  __device__ static float2 cvt(uint32_t w, int pol) {
    const uint32_t a = w >> (16 * pol);
    return make_float2((float)(int8_t)(a & 0xffu), (float)(int8_t)((a >> 8) & 0xffu));
  }
};

// Ring control, first in the shared memory of either sample width: the persistent batch kernel
// runs items of both widths through one ring, so the barriers must not move with the layout.
struct PpfCtl {
  uint64_t full[kStages];         // copy-complete barriers of the ring slots
  int slot_done[kStages];         // halves done reading a slot's current tile
  int issued[kStages];            // copies issued into each slot since the kernel began
  int abort;                      // a wait gave up: every half stops at its next tile
};

template <int BITS>
struct PpfSmem {
  using word = typename SampleIO<BITS>::word;
  static constexpr int kSlot = kTile * kN + SampleIO<BITS>::kAlign;   // a tile + alignment slack
  PpfCtl ctl;
  alignas(16) float4 gain[kN / 2];             // [k1][k2 / 2]: bandpass x delay phasor, pairs of k2
  alignas(16) float2 tw[kN];                   // [k1][p2] = exp(-2 pi i k1 p2 / 256)
  // per polarisation, two tiles of v_m[p] (132 KB); each tile buffer (258 x 128 bytes) also stages
  // its tile's output for the tensor stores, so it starts on a 128-byte boundary
  alignas(128) float2 w[kP][2][kTile][kRowV];
  alignas(16) word in[kStages][kSlot];         // input ring of dual-pol samples (64 KB int16, 32 KB int8)
};
static_assert(offsetof(PpfSmem<16>, ctl) == 0 && offsetof(PpfSmem<8>, ctl) == 0, "ring control first");
static_assert((PpfSmem<16>::kSlot * sizeof(uint2)) % 16 == 0 && (PpfSmem<8>::kSlot * sizeof(uint32_t)) % 16 == 0,
              "ring slots 16-byte aligned");
static_assert(sizeof(PpfSmem<16>) <= 232448 && sizeof(PpfSmem<8>) <= 232448, "one CTA's shared memory");
static_assert(offsetof(PpfSmem<16>, w) % 128 == 0 && offsetof(PpfSmem<8>, w) % 128 == 0 &&
                  (kTile * kRowV * sizeof(float2)) % 128 == 0 && 2 * kN * 64 <= kTile * kRowV * sizeof(float2),
              "tile buffers 128-byte aligned and large enough to stage both FP16 planes of a tile");

// Output modes: the channelised layout, the FP32 corner-turned layout, or the FP16 layout of the
// tensor-core beam former ([F*N][M/32][Kpad][P][32] with station s in rows k = 2s (re), 2s+1 (im);
// a hi plane fp16(Y) and optionally a lo plane fp16(Y - hi)).
enum PpfMode { MODE_CHAN = 0, MODE_CT32 = 1, MODE_CT16 = 2 };

struct PpfOut {
  float2 *f32;
  __half *hi, *lo;
  int kpad;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Bounded wait for the phase of the given parity; false on expiry or once another thread aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
  for (uint32_t i = 0; i < kWaitIters; ++i) {
    if (mbar_test(bar, parity)) return true;
    if (*abort_flag) return false;
    if (i > 32) __nanosleep(32);
  }
  return false;
}

// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned) from global memory into
// this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Named barrier of one half (256 threads); returns whether any of them passed `pred`.
__device__ __forceinline__ bool half_sync_any(uint32_t id, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "barrier.cta.red.or.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)pred), "r"(id), "n"(kHalf)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ void half_sync(uint32_t id) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(kHalf) : "memory");
}

// Tensor maps of the FP16 planes for the filter bank's stores: boxes of 16 spectra (one pol) x the
// two K rows of a station x 256 channels (encode_ct16_store_map).
struct PpfMaps {
  CUtensorMap hi, lo;
  CUtensorMap ct;   // FP32 corner turn [F*N][S][P][M] float2: boxes of 16 spectra x kCtTma channels
  int has_lo;
};

// Bulk tensor store of one box from this CTA's shared memory (completion tracked by bulk groups).
__device__ __forceinline__ void tma_store_4d(const CUtensorMap *map, uint32_t src, int x, int y, int z, int w) {
  asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4}], [%5];"
               ::"l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(src)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// this thread's bulk stores have finished reading shared memory / have completed
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Barriers and counters of the ring, once per kernel (thread 0; the caller synchronises).
__device__ __forceinline__ void ppf_setup(PpfCtl &c) {
  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&c.full[i], 1);
      c.slot_done[i] = 0;
      c.issued[i] = 0;
    }
    c.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
}

// After the last item, with every thread of the CTA past a barrier: a CTA that gave up waits
// (bounded) for the copies it still has in flight before its shared memory is released.
__device__ __forceinline__ void ppf_drain(PpfCtl &c) {
  if (threadIdx.x == 0 && c.abort) {
    for (int i = 0; i < kStages; ++i) {
      if (c.issued[i] == 0) continue;
      const uint32_t parity = (uint32_t)(c.issued[i] - 1) & 1u;   // the last copy into slot i
      for (uint32_t k = 0; k < kWaitIters && !mbar_test(&c.full[i], parity); ++k) __nanosleep(64);
    }
  }
}

// One work item: both polarisations of spectra [chunk * spc, (chunk + 1) * spc) of stream (s, f),
// spc a multiple of 16.  On entry every thread of the CTA is done with the previous item (if any);
// `ph` holds this thread's parity bit per ring slot.
// kTmaSt: pass 2 stages each tile's FP16 planes (all of them) or FP32 corner turn (channels
// [256 - kCtTma, 256)) in the tile's own buffer and one thread per half stores them with tensor
// stores (maps), which drain while the next tile is filtered; otherwise every thread stores its
// values directly.
// kStall: failure-detection test build, the item issues none of its input copies (its waits
// expire); launched only when the test asks for it, so the production kernels are untouched.
template <int BITS, int MODE, bool kTmaSt, bool kStall = false>
__device__ __forceinline__ void ppf_item(const Geometry &g, const typename SampleIO<BITS>::word *__restrict__ in,
                                         const typename SampleIO<BITS>::word *__restrict__ hist, const PpfOut &po,
                                         int s, int f, int chunk, int spc, PpfSmem<BITS> &sm, uint32_t &ph,
                                         const PpfMaps *maps) {
  using word = typename SampleIO<BITS>::word;
  using IO = SampleIO<BITS>;
  constexpr int kAlign = IO::kAlign;
  const int tid = threadIdx.x;
  const int pol = tid / kHalf;
  const int p = tid % kHalf;
  const long long sf = (long long)s * g.F + f;
  const int m0 = chunk * spc;
  const int m_end = min(g.M, m0 + spc);
  const int ntiles = (m_end - m0 + kTile - 1) / kTile;

  // x'[j] = x[j - d_s]; block-relative x' index j lives at extended index H - d_s + j of
  // [history (H samples) | block (T samples)].  Frames r >= -15, r < M.
  const int dsh = g.dshift[s];
  const word *hs = hist + sf * g.H;
  const word *bs = in + sf * g.T;
  const bool in16 = ((reinterpret_cast<uintptr_t>(in) & 15) == 0);
  auto gpair = [&](int r) -> uint32_t {   // this thread's sample of frame r, from global memory
    const long long e = (long long)g.H - dsh + (long long)r * kN + p;
    return (e < g.H) ? IO::pair(hs, e, pol) : IO::pair(bs, e - g.H, pol);
  };
  // A tile wholly inside the block (first sample e0 = mt N - d_s >= 0) arrives by bulk copy: the
  // 16-byte-aligned run covering it, never past the stream's end (T is a multiple of N); its
  // frames start at slot offset e0 mod kAlign.
  auto is_bulk = [&](int mt) { return in16 && (long long)mt * kN - dsh >= 0; };
  auto issue = [&](int t) {   // one thread
    if (t >= ntiles || kStall) return;
    const int mt = m0 + t * kTile;
    if (!is_bulk(mt)) return;
    const int nfr = min(kTile, m_end - mt);
    const long long e0 = (long long)mt * kN - dsh;
    const long long a = e0 & ~(long long)(kAlign - 1);
    const uint32_t bytes = (uint32_t)((e0 - a + (long long)nfr * kN + kAlign - 1) / kAlign) * 16u;
    const int st = t % kStages;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // earlier generic reads of the slot
    mbar_expect_tx(&sm.ctl.full[st], bytes);
    bulk_g2s(sm.in[st], bs + a, bytes, &sm.ctl.full[st]);
    sm.ctl.issued[st] += 1;
  };
  if (tid == 0) {
    issue(0);
    issue(1);
  }

  // per-item tables: pass-1 twiddles [k1][p2] and the epilogue gain of channel k1 + 16((k2+8)&15)
  // (FP32 corner turn only: the FP16 planes leave the delay phase and bandpass to the tensor-core
  // weights)
  if (tid < kN) {
    sm.tw[tid] = g.twiddle[(tid & 15) * (tid >> 4)];
  } else if (MODE == MODE_CT32) {
    // Y = X * bp[c] * exp(+2 pi i (f0 tau_s + df_c (tau_s - n_s Ts))), phase in FP64 cycles
    const int i = tid - kN, k1 = i >> 4, k2 = i & 15;
    const int c = k1 + 16 * ((k2 + 8) & 15);
    const double df = (double)(c - kN / 2) * (g.fs / kN);
    const double phi = g.f0[f] * g.tau[s] + df * g.resid[s];
    const float2 ph2 = unit_phasor_cycles(phi);
    const float b = g.bandpass[c];
    reinterpret_cast<float2 *>(sm.gain)[i] = make_float2(b * ph2.x, b * ph2.y);
  }

  float2 h2[kL];   // (h, h): one packed FMA updates both components
#pragma unroll
  for (int t = 0; t < kL; ++t) {
    const float hv = g.taps[t * kN + p];
    h2[t] = make_float2(hv, hv);
  }
  float2 win[kL];   // frame r of this polarisation is kept in slot r & 15 (m0 is a multiple of 16)
#pragma unroll
  for (int i = 0; i < kL - 1; ++i) win[i + 1] = IO::cvt(gpair(m0 - (kL - 1) + i), pol);
  __syncthreads();   // tables

  // this half's two FIR buffers: tile t lives in wbuf[t & 1] (FIR output, transformed in place by
  // pass 1, read by pass 2)
  float2(*wbuf)[kTile][kRowV] = sm.w[pol];
  const uint32_t bar_x = 1 + pol, bar_y = 1 + kP + pol;   // this half's named barriers
  const uint32_t bar_z = 1 + 2 * kP + pol, bar_w = 1 + 3 * kP + pol;   // pass 2 staging (kTmaSt)
  const int m1 = p >> 4, c1 = p & 15;   // pass-1 thread: spectrum m1, column p2 = c1
  const int m2 = p & 15, k1 = p >> 4;   // pass-2 thread: spectrum m2, row segment k1

  // wait for tile t's copy (bulk tiles only); false if this thread's wait gave up
  auto wait_tile = [&](int t) -> bool {
    if (!is_bulk(m0 + t * kTile)) return true;
    const int st = t % kStages;
    const bool ok = mbar_wait(&sm.ctl.full[st], (ph >> st) & 1u, &sm.ctl.abort);
    ph ^= 1u << st;
    if (!ok && atomicExch(&sm.ctl.abort, 1) == 0 && g.err) atomicCAS(g.err, 0, DERR_PPF_INPUT);
    return ok;
  };
  // this half is done reading tile t's slot: the second half to get here refills it with t + 2
  auto release_slot = [&](int t) {
    const int st = t % kStages;
    if (p == 0 && atomicAdd(&sm.ctl.slot_done[st], 1) == kP - 1) {
      atomicExch(&sm.ctl.slot_done[st], 0);
      issue(t + kStages);
    }
  };
  auto aborted = [&]() { return *reinterpret_cast<volatile int *>(&sm.ctl.abort) != 0; };

  // FIR outputs [Q0, Q1) of tile t into wbuf[t & 1]:
  // v_m[p] = sum_t h[tN + p] x'[(m - 15 + t) N + p], this polarisation
  auto fir = [&](int t, auto q0c, auto q1c, auto fullc, auto directc) {
    constexpr int Q0 = decltype(q0c)::value, Q1 = decltype(q1c)::value;
    constexpr bool kFull = decltype(fullc)::value, kDirect = decltype(directc)::value;
    const int mt = m0 + t * kTile;
    const int nfr = min(kTile, m_end - mt);
    const long long e0 = (long long)mt * kN - dsh;
    const word *slot = sm.in[t % kStages] + (kDirect ? 0 : (int)(e0 & (kAlign - 1))) + p;
    float2 *vout = &wbuf[t & 1][0][p];
#pragma unroll
    for (int q = Q0; q < Q1; ++q) {
      if (kFull || q < nfr)
        win[q] = IO::cvt(kDirect ? gpair(mt + q) : IO::pair(slot, (long long)q * kN, pol), pol);
      else
        win[q] = make_float2(0.f, 0.f);
      // two partial sums per component halve the FMA dependency chain
      float2 acc = __fmul2_rn(h2[0], win[(q + 1) & 15]);
      float2 acc1 = __fmul2_rn(h2[1], win[(q + 2) & 15]);
#pragma unroll
      for (int tap = 2; tap < kL; tap += 2) {
        acc = __ffma2_rn(h2[tap], win[(q + 1 + tap) & 15], acc);
        acc1 = __ffma2_rn(h2[tap + 1], win[(q + 2 + tap) & 15], acc1);
      }
      vout[q * kRowV] = __fadd2_rn(acc, acc1);
    }
  };
  // call body(full, direct) with the FIR variant of tile t as compile-time flags
  auto with_variant = [&](int t, auto &&body) {
    const int mt = m0 + t * kTile;
    const bool full = m_end - mt >= kTile, bulk = is_bulk(mt);
    if (bulk && full) body(std::true_type(), std::false_type());
    else if (bulk) body(std::false_type(), std::false_type());
    else if (full) body(std::true_type(), std::true_type());
    else body(std::false_type(), std::true_type());
  };

  // ---- FFT pass 1 of tile t, in place: column p2 = c1 of spectrum m1, 16-point DFT over p1,
  // twiddle W256^(p2 k1); the thread reads and writes only its own 16 points
  auto pass1 = [&](int t) {
    float2 *col = &wbuf[t & 1][m1][c1];
    float2 a[16];
#pragma unroll
    for (int p1 = 0; p1 < 16; ++p1) a[p1] = col[16 * p1];
    dft16(a);
    col[0] = a[0];
#pragma unroll
    for (int k = 1; k < 16; ++k) col[16 * k] = cmul(a[k], sm.tw[16 * k + c1]);
  };

  // ---- FFT pass 2 of tile t: row segment k1 of spectrum m2, 16-point DFT over p2:
  // a[k2] = X[k1 + 16 k2], channel c = (k + N/2) mod N = k1 + 16 ((k2 + 8) & 15)
  // fullc (FP16 planes with tensor stores): a full tile, no spectrum past the block's end to zero
  auto pass2 = [&](int t, auto fullc) {
    constexpr bool kFullTile = decltype(fullc)::value;
    const int mt = m0 + t * kTile;
    float2 a[16];
    const float4 *src = reinterpret_cast<const float4 *>(&wbuf[t & 1][m2][16 * k1]);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float4 v = src[i];
      a[2 * i] = make_float2(v.x, v.y);
      a[2 * i + 1] = make_float2(v.z, v.w);
    }
    if constexpr (MODE != MODE_CHAN && kTmaSt) half_sync(bar_z);   // the buffer is read: staging may overwrite it
    dft16(a);
    const int mg = mt + m2;
    if (MODE == MODE_CHAN) {
      if (mg < m_end) {
        float2 *dst = po.f32 + ((((long long)f * g.S + s) * kP + pol) * g.M + mg) * kN + k1;
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) dst[16 * ((k2 + 8) & 15)] = a[k2];
      }
    } else {
      if (MODE == MODE_CT32) {
        const float4 *gp = &sm.gain[k1 * 8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float4 gg = gp[i];
          a[2 * i] = cmul(a[2 * i], make_float2(gg.x, gg.y));
          a[2 * i + 1] = cmul(a[2 * i + 1], make_float2(gg.z, gg.w));
        }
        // ct[f][c][s][pol][m]: the 16 lanes of a channel write 16 consecutive spectra (128 B)
        if constexpr (kTmaSt) {
          // channel c = k1 + 16 j (j = (k2 + 8) & 15): j >= 16 - kCtTma / 16 goes to the staging
          // box [kCtTma channels][16 spectra] float2, the rest straight to global memory
          constexpr int kJ0 = 16 - kCtTma / 16;
          unsigned char *stg = reinterpret_cast<unsigned char *>(&wbuf[t & 1][0][0]) + kCtStageOff;
          float2 *dst = po.f32 + ((((long long)f * kN + k1) * g.S + s) * kP + pol) * g.M + mg;
          const long long cstep = 16LL * g.S * kP * g.M;
#pragma unroll
          for (int k2 = 0; k2 < 16; ++k2) {
            const int j = (k2 + 8) & 15;
            if (j >= kJ0)
              *reinterpret_cast<float2 *>(stg + ((j - kJ0) * 16 + k1) * 128 + m2 * 8) = a[k2];
            else if (mg < m_end)
              dst[j * cstep] = a[k2];
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // staging visible to the tensor store
          half_sync(bar_w);
          if (p == 0) {
            tma_store_4d(&maps->ct, smem_u32(stg), 2 * mt, pol, s, f * kN + kN - kCtTma);
            bulk_commit();
          }
          return;
        }
        if (mg < m_end) {
          float2 *dst = po.f32 + ((((long long)f * kN + k1) * g.S + s) * kP + pol) * g.M + mg;
          const long long cstep = 16LL * g.S * kP * g.M;
#pragma unroll
          for (int k2 = 0; k2 < 16; ++k2) dst[((k2 + 8) & 15) * cstep] = a[k2];
        }
      } else {
        // [F*N][Mt][Kpad][P][32] halves, rows k = 2s (re) and 2s+1 (im).  Lanes m and m^1 swap
        // halves of their value: the even lane then holds Re of spectra (m, m+1), the odd lane
        // Im of (m-1, m), each written as one half2 per plane.  Spectra at or past the block's
        // end go out as zeros (pad columns of the last tile).
        const int odd = m2 & 1;
        const int me = mg & ~1;
        const bool v0 = me < m_end, v1 = me + 1 < m_end;
        if constexpr (kTmaSt) {
          // staging = the tensor store's box: [256 channels][row 2s, 2s+1][16 spectra] halves per
          // plane (64 bytes per channel), hi plane then lo plane, in this tile's buffer
          unsigned char *stg = reinterpret_cast<unsigned char *>(&wbuf[t & 1][0][0]);
          const int col = odd * 32 + (m2 & ~1) * 2;
#pragma unroll
          for (int k2 = 0; k2 < 16; ++k2) {
            const float send = odd ? a[k2].x : a[k2].y;
            const float recv = __shfl_xor_sync(0xffffffffu, send, 1);
            float2 x = make_float2(odd ? recv : a[k2].x, odd ? a[k2].y : recv);
            if (!kFullTile) {
              if (!v0) x.x = 0.f;
              if (!v1) x.y = 0.f;
            }
            const __half2 h = __floats2half2_rn(x.x, x.y);
            const float2 lo = sub2(x, __half22float2(h));   // exact: x - hi
            const int o = (k1 + 16 * ((k2 + 8) & 15)) * 64 + col;
            *reinterpret_cast<__half2 *>(stg + o) = h;
            *reinterpret_cast<__half2 *>(stg + 16384 + o) = __floats2half2_rn(lo.x, lo.y);
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // staging visible to the tensor stores
          if (p == 0) bulk_wait_read();   // the previous tile's stores have read their staging
          half_sync(bar_w);
          if (p == 0) {
            const uint32_t src = smem_u32(stg);
            tma_store_4d(&maps->hi, src, pol * 32 + (mt & 31), 2 * s, mt >> 5, f * kN);
            if (maps->has_lo) tma_store_4d(&maps->lo, src + 16384, pol * 32 + (mt & 31), 2 * s, mt >> 5, f * kN);
            bulk_commit();
          }
          return;
        }
        const int mb = tc_tiles(g.M);
        const long long rowbase = (long long)(me >> 5) * po.kpad + 2 * s + odd;
        const long long cstride = (long long)mb * po.kpad * 64;
        __half *hi0 = po.hi + (((long long)f * kN + k1) * mb * po.kpad + rowbase) * 64 + pol * 32 + (me & 31);
        __half *lo0 = po.lo ? po.lo + (hi0 - po.hi) : nullptr;
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) {
          const float send = odd ? a[k2].x : a[k2].y;
          const float recv = __shfl_xor_sync(0xffffffffu, send, 1);
          float x0 = odd ? recv : a[k2].x;
          float x1 = odd ? a[k2].y : recv;
          if (!v0) x0 = 0.f;
          if (!v1) x1 = 0.f;
          const __half2 h = __floats2half2_rn(x0, x1);
          const float2 hf = __half22float2(h);
          const long long o = (long long)(16 * ((k2 + 8) & 15)) * cstride;
          *reinterpret_cast<__half2 *>(hi0 + o) = h;
          if (lo0) *reinterpret_cast<__half2 *>(lo0 + o) = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
        }
      }
    }
  };

  using I0 = std::integral_constant<int, 0>;
  using I8 = std::integral_constant<int, kTile / 2>;
  using I16 = std::integral_constant<int, kTile>;
  // Software pipeline: the FIR of tile t + 1 runs inside the FFT phases of tile t, so every warp
  // has independent FMA work to issue while its shared-memory loads are in flight.  Direct stores:
  //   prologue:  FIR(0)                               | barrier x
  //   tile t:    pass 1(t) + FIR(t + 1) outputs 0..7  | barrier x (pass 1 done; abort check)
  //              pass 2(t) + FIR(t + 1) outputs 8..15 | barrier y (wbuf[t & 1] free, FIR done)
  // With tensor stores (kFirA = 0) the whole FIR of tile t + 1 runs in the pass-2 phase, which
  // stages tile t in wbuf[t & 1] between barriers z and w; before barrier x thread 0 of the half
  // waits until the store of tile t - 1 has read wbuf[(t + 1) & 1], which that FIR refills.
  // The FP16-plane output keeps its pass 2 (shuffles and the hi/lo split) apart from the FIR: the
  // pipelined schedule measured 8 % slower for it (spilling with 16-bit samples, and slower
  // without spills with 8-bit ones).  Its schedule is sequential over the same two buffers:
  //   tile t:    FIR(t) | barrier x (slot free) | pass 1(t) | barrier y | pass 2(t) loads |
  //              barrier z (buffer read) | staging | barrier w | tensor stores of tile t
  // (thread 0 of the half waits, before barrier w, until the stores of tile t - 1 have read their
  // buffer, which FIR(t + 1) refills next)
  if constexpr (MODE == MODE_CT16) {
    for (int t = 0; t < ntiles; ++t) {
      const bool failed = !wait_tile(t);
      with_variant(t, [&](auto full, auto direct) { fir(t, I0(), I16(), full, direct); });
      if (half_sync_any(bar_x, failed || aborted())) return;
      release_slot(t);
      pass1(t);
      half_sync(bar_y);
      if (m_end - (m0 + t * kTile) >= kTile) pass2(t, std::true_type());
      else pass2(t, std::false_type());
    }
    // the last tile's stores have read their buffer before another item's FIR refills it
    if (kTmaSt && p == 0) bulk_wait_read();
    return;
  }
  {
    const bool failed = !wait_tile(0);
    with_variant(0, [&](auto full, auto direct) { fir(0, I0(), I16(), full, direct); });
    if (half_sync_any(bar_x, failed || aborted())) return;
    release_slot(0);
  }
  using IA = std::integral_constant<int, kTmaSt ? kFirA : kTile / 2>;
  for (int t = 0; t < ntiles; ++t) {
    const bool next = t + 1 < ntiles;
    const bool failed = next && !wait_tile(t + 1);
    if (next)
      with_variant(t + 1, [&](auto full, auto direct) {
        pass1(t);
        fir(t + 1, I0(), IA(), full, direct);
      });
    else
      pass1(t);
    // the tensor store of tile t - 1 has read its staging rows, which the FIR of tile t + 1 below
    // (inside pass 2) refills
    if (kTmaSt && p == 0) bulk_wait_read();
    if (half_sync_any(bar_x, failed || aborted())) return;
    if (next)
      with_variant(t + 1, [&](auto full, auto direct) {
        pass2(t, std::false_type());
        fir(t + 1, IA(), I16(), full, direct);
      });
    else
      pass2(t, std::false_type());
    half_sync(bar_y);
    if (next) release_slot(t + 1);
  }
  if (kTmaSt && p == 0) bulk_wait_read();   // as above
}

template <int BITS, int MODE, bool kTma, bool kStall = false>
__global__ void __launch_bounds__(kThreads, 1)
ppf_kernel(Geometry g, const typename SampleIO<BITS>::word *__restrict__ in,
           const typename SampleIO<BITS>::word *__restrict__ hist, PpfOut po, int chunks, int spc,
           const __grid_constant__ PpfMaps maps) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // The tensor stores read 128-byte-aligned staging buffers: the layout aligns them within itself
  // and the base is declared 128-byte aligned (this kernel has no static shared memory).  Rounding
  // the base up at run time instead cost the FP32 form registers (spills); a base that is not
  // aligned after all is reported (device error 5) and the CTA writes nothing.
  if (kTma && (smem_u32(smem_raw) & 127u) != 0) {
    if (threadIdx.x == 0 && g.err) atomicCAS(g.err, 0, DERR_PPF_ALIGN);
    return;
  }
  PpfSmem<BITS> &sm = *reinterpret_cast<PpfSmem<BITS> *>(smem_raw);
  int s, f, chunk;
  const long long item = blockIdx.x;
  if (MODE == MODE_CT16) {   // stations fastest: neighbouring CTAs fill neighbouring K rows of the
    s = (int)(item % g.S);   // same (channel) planes
    const long long rest = item / g.S;
    chunk = (int)(rest % chunks);
    f = (int)(rest / chunks);
  } else {
    const long long sf = item / chunks;          // stream index s * F + f
    chunk = (int)(item - sf * chunks);
    s = (int)(sf / g.F);
    f = (int)(sf - (long long)s * g.F);
  }
  ppf_setup(sm.ctl);
  uint32_t ph = 0;
  if (kStall && item == g.ppf_stall)
    ppf_item<BITS, MODE, kTma, true>(g, in, hist, po, s, f, chunk, spc, sm, ph, &maps);
  else
    ppf_item<BITS, MODE, kTma>(g, in, hist, po, s, f, chunk, spc, sm, ph, &maps);
  // the tensor stores of the last tiles complete (read and written) before the CTA's shared
  // memory is released; only thread 0 of each half issued any
  if (kTma && threadIdx.x % kHalf == 0) bulk_wait_all();
  __syncthreads();
  ppf_drain(sm.ctl);
}

// Persistent filter bank over the blocks of several observations (a batch): CTAs take work items
// (stream, spectrum chunk: both polarisations) from a shared counter until all groups are done.
// One launch per class of sample width and output form, so each body keeps the registers it has
// when its observation runs alone.  The observations' geometry comes in a grid-constant table
// (constant bank); thread 0 finds each item's observation.
template <int BITS, int MODE, bool kTma>
__global__ void __launch_bounds__(kThreads, 1)
ppf_group_kernel(const __grid_constant__ PpfTable T, long long total, unsigned long long *counter) {
  using word = typename SampleIO<BITS>::word;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ long long item_s;
  __shared__ int grp_s;
  if (kTma && (smem_u32(smem_raw) & 127u) != 0) {   // staging buffers must be 128-byte aligned
    if (threadIdx.x == 0 && T.grp[0].g.err) atomicCAS(T.grp[0].g.err, 0, DERR_PPF_ALIGN);
    return;
  }
  PpfSmem<BITS> &sm = *reinterpret_cast<PpfSmem<BITS> *>(smem_raw);
  ppf_setup(sm.ctl);
  uint32_t ph = 0;
  // thread 0 takes the next item while the current one runs (the counter's latency stays hidden)
  long long nxt = threadIdx.x == 0 ? (long long)atomicAdd(counter, 1ull) : 0;
  for (;;) {
    if (threadIdx.x == 0) {
      const long long it = sm.ctl.abort ? total : nxt;
      item_s = it;
      grp_s = it < total ? group_of(T, it) : 0;
      if (it < total) nxt = (long long)atomicAdd(counter, 1ull);
    }
    __syncthreads();
    const long long item = item_s;
    const int o = grp_s;
    __syncthreads();
    if (item >= total) break;
    const PpfGroup &G = T.grp[o];
    const long long local = item - G.first_item;
    const long long sf = local / G.chunks;
    const int chunk = (int)(local - sf * G.chunks);
    const int s = (int)(sf / G.g.F), f = (int)(sf - (long long)s * G.g.F);
    const PpfOut po = MODE == MODE_CT16
        ? PpfOut{nullptr, reinterpret_cast<__half *>(G.ct16.hi), reinterpret_cast<__half *>(G.ct16.lo), G.ct16.kpad}
        : PpfOut{G.ct, nullptr, nullptr, 0};
    ppf_item<BITS, MODE, kTma>(G.g, (const word *)G.in, (const word *)G.hist, po, s, f, chunk, G.spc, sm, ph,
                               kTma ? static_cast<const PpfMaps *>(G.maps) : nullptr);
  }
  if (kTma && threadIdx.x % kHalf == 0) bulk_wait_all();
  __syncthreads();
  ppf_drain(sm.ctl);
}

template <int BITS, int MODE, bool kTma>
cudaError_t launch_group_t(const PpfTable &T, long long total, unsigned long long *counter, int ctas,
                           cudaStream_t st) {
  const size_t smem = sizeof(PpfSmem<BITS>);
  auto kern = ppf_group_kernel<BITS, MODE, kTma>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  kern<<<ctas, kThreads, smem, st>>>(T, total, counter);
  return cudaGetLastError();
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

template <int BITS, int MODE, bool kTma>
cudaError_t launch_ppf_t(const Geometry &g, const void *in, const void *hist, PpfOut po, const PpfMaps &maps,
                         cudaStream_t st) {
  using word = typename SampleIO<BITS>::word;
  const long long streams = (long long)g.S * g.F;   // one CTA: both polarisations
  if (streams == 0 || g.M == 0) return cudaSuccess;
  const long long want = (kMinCtas + streams - 1) / streams;      // chunks per stream wanted
  const int spc = (int)((((long long)g.M + want - 1) / want + kTile - 1) / kTile) * kTile;
  const int chunks = (g.M + spc - 1) / spc;
  const long long ctas = streams * chunks;
  if (ctas == 0) return cudaSuccess;
  const size_t smem = sizeof(PpfSmem<BITS>);
  auto go = [&](auto kern) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)ctas, kThreads, smem, st>>>(g, (const word *)in, (const word *)hist, po, chunks, spc, maps);
    return cudaGetLastError();
  };
  // the failure-detection test build (FP32 corner turn only) when one CTA is to stall
  if constexpr (MODE == MODE_CT32)
    if (g.ppf_stall >= 0 && g.ppf_stall < ctas) return go(ppf_kernel<BITS, MODE, kTma, true>);
  return go(ppf_kernel<BITS, MODE, kTma>);
}

template <int BITS>
cudaError_t launch_ppf_bits(const Geometry &g, const void *in, const void *hist, float2 *chan, float2 *ct,
                            const Ct16Out *ct16, cudaStream_t st) {
  PpfOut po{nullptr, nullptr, nullptr, 0};
  PpfMaps maps{};
  if (ct16) {
    po.hi = reinterpret_cast<__half *>(ct16->hi);
    po.lo = reinterpret_cast<__half *>(ct16->lo);
    po.kpad = ct16->kpad;
    if ((long long)g.S * g.F == 0 || g.M == 0) return cudaSuccess;
    const long long fc_rows = (long long)g.F * kN;
    cudaError_t e = encode_ct16_store_map(&maps.hi, ct16->hi, ct16->kpad, g.M, fc_rows);
    if (e == cudaSuccess && ct16->lo) e = encode_ct16_store_map(&maps.lo, ct16->lo, ct16->kpad, g.M, fc_rows);
    if (e != cudaSuccess) return e;
    maps.has_lo = ct16->lo != nullptr;
    return launch_ppf_t<BITS, MODE_CT16, true>(g, in, hist, po, maps, st);
  }
  if (ct) {
    po.f32 = ct;
    // a tensor map over [F*N][S][P][M] float2 needs 16-byte strides (M even) and base
    if ((long long)g.S * g.F > 0 && g.M > 0 && g.M % 2 == 0 && (reinterpret_cast<uintptr_t>(ct) & 15) == 0) {
      cudaError_t e = encode_ct32_store_map(&maps.ct, ct, g.S, g.M, (long long)g.F * kN, kCtTma);
      if (e != cudaSuccess) return e;
      return launch_ppf_t<BITS, MODE_CT32, true>(g, in, hist, po, maps, st);
    }
    return launch_ppf_t<BITS, MODE_CT32, false>(g, in, hist, po, maps, st);
  }
  po.f32 = chan;
  return launch_ppf_t<BITS, MODE_CHAN, false>(g, in, hist, po, maps, st);
}

}  // namespace

int ppf_items_per_stream(int M, int spc) { return (M + spc - 1) / spc; }
int ppf_ctas_per_sm() { return 1; }

cudaError_t launch_ppf(const Geometry &g, int bits, const void *in, const void *hist, float2 *chan,
                       float2 *ct, cudaStream_t st, const Ct16Out *ct16) {
  return bits == 16 ? launch_ppf_bits<16>(g, in, hist, chan, ct, ct16, st)
                    : launch_ppf_bits<8>(g, in, hist, chan, ct, ct16, st);
}

bool ppf_group_tma(const PpfGroup &G) {
  if ((long long)G.g.S * G.g.F == 0 || G.g.M == 0) return false;
  if (G.tc) return true;
  return G.g.M % 2 == 0 && (reinterpret_cast<uintptr_t>(G.ct) & 15) == 0;
}

size_t ppf_group_maps_bytes() { return sizeof(PpfMaps); }

cudaError_t ppf_group_maps(const PpfGroup &G, void *host_dst) {
  if (!ppf_group_tma(G)) return cudaErrorInvalidValue;
  PpfMaps m{};
  const long long fc_rows = (long long)G.g.F * kN;
  cudaError_t e;
  if (G.tc) {
    e = encode_ct16_store_map(&m.hi, G.ct16.hi, G.ct16.kpad, G.g.M, fc_rows);
    if (e == cudaSuccess && G.ct16.lo) e = encode_ct16_store_map(&m.lo, G.ct16.lo, G.ct16.kpad, G.g.M, fc_rows);
    m.has_lo = G.ct16.lo != nullptr;
  } else {
    e = encode_ct32_store_map(&m.ct, G.ct, G.g.S, G.g.M, fc_rows, kCtTma);
  }
  if (e == cudaSuccess) std::memcpy(host_dst, &m, sizeof(m));
  return e;
}

cudaError_t launch_ppf_group(int bits, int tc, int tma, const PpfGroup *h_groups, int ngrp, long long total,
                             unsigned long long *counter, int ctas, cudaStream_t st) {
  if (total == 0) return cudaSuccess;
  if (ngrp < 1 || ngrp > kMaxGroups) return cudaErrorInvalidValue;
  PpfTable T;
  T.n = ngrp;
  for (int i = 0; i < ngrp; ++i) T.grp[i] = h_groups[i];
  if (tma) {
    if (bits == 16) return tc ? launch_group_t<16, MODE_CT16, true>(T, total, counter, ctas, st)
                              : launch_group_t<16, MODE_CT32, true>(T, total, counter, ctas, st);
    return tc ? launch_group_t<8, MODE_CT16, true>(T, total, counter, ctas, st)
              : launch_group_t<8, MODE_CT32, true>(T, total, counter, ctas, st);
  }
  if (bits == 16) return tc ? launch_group_t<16, MODE_CT16, false>(T, total, counter, ctas, st)
                            : launch_group_t<16, MODE_CT32, false>(T, total, counter, ctas, st);
  return tc ? launch_group_t<8, MODE_CT16, false>(T, total, counter, ctas, st)
            : launch_group_t<8, MODE_CT32, false>(T, total, counter, ctas, st);
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
