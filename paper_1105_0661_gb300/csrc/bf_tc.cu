// Tensor-core tied-array beam former (Section 4.3) for many beams: tcgen05 UMMA with FP16 operands
// and FP32 accumulation in TMEM, fused with the Stokes I / IQUV integration epilogue (Sections 4.5,
// 5.1) or writing the beam voltages (complex-voltage output, Section 3).
//
// Per (subband f, channel c) the complex product V = W Y is run as a real GEMM
//     D[r][n] = sum_k A[r][k] B[k][n],   r = (beam, re|im),  k = (station, re|im),  n = (pol, m)
// with A rows (Re w, -Im w) / (Im w, Re w): D[2b] = Re V_b, D[2b+1] = Im V_b.  Both operands are
// split into FP16 hi and lo = fp16(x - hi) parts; the products Whi Yhi + Wlo Yhi + Whi Ylo
// accumulate in FP32 into the same TMEM tile, which keeps the error at the level of the FP32 path
// rather than of FP16 rounding (the filtered spectrum Y is not exact in FP16 for either sample
// width, and beams summed with cancellation magnify its rounding).  The two-product form drops
// Wlo Yhi: FP16 weights (rounding error <= 2^-12 per component) against the hi+lo spectrum, two
// thirds of the MMA work.
//
// Operands.  A (the weights) lives in tensor memory: the epilogue warps compute it from the
// FP64-reduced phase tables with the hardware sincos of the reduced phase and write it with
// tcgen05.st, one TMEM lane per row, two FP16 K elements per 32-bit column.  B is the filter
// bank's FP16 scratch
// [F*N][Mt][Kpad][P][32] (Mt = ceil(M/64)*2 tiles of 32 spectra; k = 2 station + re|im; a 128-byte
// row holds the 2 pols x 32 spectra of one k), brought into shared memory by TMA two tiles at a
// time (one box of 2 x Kpad rows per plane, 128-byte swizzle) and read by the MMA as an MN-major
// operand of N = 128 columns: two 64-column swizzle atoms, Kpad x 128 bytes apart.
//
// Work.  A persistent CTA per SM walks the work items (f, c, block of 128 beams) with a stride of
// the grid, so the CTAs that run together share the (f, c) B tiles in L2.  An item is two UMMA M
// tiles of 128 rows (64 beams each) by ceil(M/64) N tiles.  Warp roles: warp 0 issues the TMA
// loads into a ring of stages, warp 1 issues the MMAs (M 128 x N 128 x K 16), the other warps are
// the epilogue: warp w serves the TMEM lane quadrant w%4 of both M tiles, 2 or 4 warps per
// quadrant (epi_split), each draining its share of the spectra of every accumulator.  Each M tile
// has one accumulator of 128 columns; the two tiles ping-pong, so that the epilogue drains one
// while the MMAs fill the other.  The epilogue warps of an M tile write its next item's weights as
// soon as the MMAs that read the weights they replace are complete: at the item's last tile pair
// with one weight set (three products), at its first with two (the two-product form).
//
// The epilogue integrates each polarisation component over the window in registers (one shuffle
// per spectrum for Stokes V) and combines the (Re, Im) row pair with two shuffles per window.
// Every mbarrier wait is bounded: on expiry the kernel records an error code, stops issuing work,
// waits (bounded) for its own copies and MMAs in flight, frees TMEM and returns.
#include <cuda.h>
#include <cuda_fp16.h>

#include "lbf_internal.cuh"

namespace lbf {
namespace {

constexpr int kRows = 128;                  // UMMA M
constexpr int kMTiles = 2;                  // 128 beams per work item
constexpr int kBeamsPerItem = kMTiles * kRows / 2;
constexpr int kSpec = 32;                   // spectra per scratch tile (one 64-column atom)
constexpr int kCols = 4 * kSpec;            // UMMA N: two tiles x (pol X, pol Y) x 32 spectra
constexpr int kMaxKpad = 128;               // S <= 64
constexpr int kMaxStages = 8;
constexpr int kBarBytes = 1024;             // barriers, TMEM slot, flags
constexpr int kSmemLimit = 227 * 1024;
constexpr int kRingBytes = kSmemLimit - 1024 /* alignment slack */ - kBarBytes;
constexpr int kMinSmem = 120 * 1024;
constexpr uint32_t kTmemCols = 512;         // 2 accumulators of 128 + 2 x 2 weight planes of <= 64
constexpr uint32_t kAccCols = kCols;
constexpr uint32_t kACol0 = kMTiles * kAccCols;   // first weight column (wcol)
constexpr uint32_t kWaitIters = 1u << 20;

// Epilogue warps per TMEM lane quadrant: 4 for Stokes outputs whose windows fit in 16 spectra (each
// warp drains 16 spectra of an accumulator), else 2 (32 spectra each).  The epilogue is the longer
// side of a work item, so more warps per accumulator shorten it.
template <int NS, int Q>
__host__ __device__ constexpr int epi_split() { return (NS != 0 && Q <= 16) ? 4 : 2; }
template <int NS, int Q>
__host__ __device__ constexpr int tc_threads() { return 64 + 4 * 32 * epi_split<NS, Q>(); }

enum ErrCode { ERR_NONE = 0, ERR_PRODUCER = 1, ERR_MMA = 2, ERR_EPILOGUE = 3 };

// One plan of a launch.
struct TcParams {
  int S, F, B, M, Kpad, ntiles, items_per_fc;
  int items;                  // F * 256 * items_per_fc (< 2^31 for any plan that fits in memory)
  int first_item;             // the plan's first work item in the launch
  int stage_bytes;            // its ring stage: 2 planes x 2 tiles x Kpad K rows x 128 bytes
  int vec;                    // output rows 16-byte aligned (M/Q % 4 == 0, aligned base)
  int wlo;                    // 1: three products (Wlo Yhi too); 0: two products
  const float *phase0, *step;
  const float *bp;            // bandpass applied to the outputs (raw FP16 planes), or null
  float *out;
  int *err;                   // the plan's device error word
};

// A launch: up to kMaxPlans plans of the same output kind and integration length, whose work
// items are numbered one after the other, so that one persistent grid walks all of them (a batch
// of uneven observations shares the SMs).  The TMA descriptors of plan i are map[2i] (hi plane)
// and map[2i + 1] (lo plane); the whole table is a grid-constant kernel parameter.
constexpr int kMaxPlans = 32;
struct TcLaunch {
  CUtensorMap map[2 * kMaxPlans];
  TcParams plan[kMaxPlans];
  int nplans, items;          // plans, and work items of all plans
  int nstages, stage_max;     // ring stages, sized for the plan with the largest stage
  long long stall_item;       // failure-detection test: the loads stop at this item (-1: never)
};

__device__ __forceinline__ int plan_of(const TcLaunch &L, int item) {
  int i = 0;
  while (i + 1 < L.nplans && L.plan[i + 1].first_item <= item) ++i;
  return i;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Bounded wait for the phase with the given parity; false on expiry or when another role aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag) {
  for (uint32_t i = 0; i < kWaitIters; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (*abort_flag) return false;
    if (i > 64) __nanosleep(64);
  }
  return false;
}

__device__ __forceinline__ void fail(volatile int *abort_flag, int *err, int code) {
  *abort_flag = 1;
  atomicCAS(err, 0, code);
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int x, int y, int z, int w,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(bar)
      : "memory");
}

// UMMA shared-memory descriptor of the MN-major B operand with the 128-byte swizzle: atoms of 8 K
// rows x 128 bytes; the next 8 K rows are 1024 bytes on (stride offset), the next 64 columns
// `lbo` bytes on (leading offset).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;                       // descriptor version
  d |= (uint64_t)2 << 61;                       // SWIZZLE_128B
  return d;
}

// Instruction descriptor: kind::f16, D = F32, A = B = F16, A K-major, B MN-major, M = 128, N = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 16) | ((uint32_t)(kCols >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);

// D[tmem] (+)= A[tmem] B[smem]
__device__ __forceinline__ void umma(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}"
      ::"r"(d_tmem), "r"(a_tmem), "l"(b), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
               ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
               : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_half2(float lo_k, float hi_k) {
  const __half2 h = __floats2half2_rn(lo_k, hi_k);   // .x (low 16 bits) is the lower K index
  return *reinterpret_cast<const uint32_t *>(&h);
}

// Weights of this thread's A row for work item (f, c) into its TMEM lane: column s of plane hi/lo
// holds (Re w, -Im w) for a Re row and (Im w, Re w) for an Im row.  The two lanes of a beam each
// evaluate every other station and swap the results; the KS warps of a lane quadrant take every
// KS-th group of 8 columns (`half` = the warp's index in its quadrant).  The phase-table values
// are loaded first (load_weight_tables), so that their latency hides behind an accumulator wait.
// With KS warps per quadrant, warp `sub` takes the groups of 8 columns g8 = sub (mod KS).
template <int KS>
struct WeightTables {
  static constexpr int kN8 = kMaxKpad / 16 / KS;   // groups of 8 stations per warp
  static constexpr int kSt = 4 * kN8;              // stations one thread evaluates per M tile
  float ph[kSt], st[kSt];   // FP64-reduced phase of the subband, phase step per channel
  uint32_t ok;              // bit i: station i of this thread exists (else weight 0)
};

template <int KS>
__device__ __forceinline__ void load_weight_tables(const TcParams &p, int f, int b, int ro, int half,
                                                   WeightTables<KS> &w) {
  w.ok = 0;
#pragma unroll
  for (int i = 0; i < WeightTables<KS>::kSt; ++i) {
    const int s = (half + KS * (i >> 2)) * 8 + 2 * (i & 3) + ro;
    const bool ok = b < p.B && s < p.S;
    const long long bs = (long long)b * p.S + s;
    w.ph[i] = ok ? __ldg(&p.phase0[(long long)f * p.B * p.S + bs]) : 0.f;
    w.st[i] = ok ? __ldg(&p.step[bs]) : 0.f;
    w.ok |= (ok ? 1u : 0u) << i;
  }
}

template <int KS>
__device__ __forceinline__ void write_weights(const TcParams &p, uint32_t ta_hi, uint32_t ta_lo, int c, int ro,
                                              int half, const WeightTables<KS> &tab, bool wlo) {
  const float dc = (float)(c - kN / 2);
#pragma unroll
  for (int gi = 0; gi < WeightTables<KS>::kN8; ++gi) {
    const int g8 = half + KS * gi;                   // 8 stations per store
    if (g8 >= p.Kpad / 16) break;
    uint32_t vh[8], vl[8];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int i = gi * 4 + j;
      float2 w = make_float2(0.f, 0.f);
      if ((tab.ok >> i) & 1u) {
        // phase in cycles, reduced to [-1/2, 1/2] (exact in FP32), then the hardware sine and
        // cosine of |x| <= pi: absolute error ~4e-7, twice the resolution of the hi+lo weight
        // and far below the 1e-3 bar of this path
        float phi = fmaf(dc, tab.st[i], tab.ph[i]);
        phi -= rintf(phi);
        __sincosf(6.283185307179586f * phi, &w.y, &w.x);
      }
      float2 o;
      o.x = __shfl_xor_sync(0xffffffffu, w.x, 1);
      o.y = __shfl_xor_sync(0xffffffffu, w.y, 1);
#pragma unroll
      for (int e = 0; e < 2; ++e) {      // station 2j + e of the group
        const float2 ws = (e == ro) ? w : o;
        const __half2 hh = __floats2half2_rn(ws.x, ws.y);
        const float2 hf = __half22float2(hh);
        const float lx = ws.x - hf.x, ly = ws.y - hf.y;
        vh[2 * j + e] = ro ? pack_half2(hf.y, hf.x) : pack_half2(hf.x, -hf.y);
        vl[2 * j + e] = ro ? pack_half2(ly, lx) : pack_half2(lx, -ly);
      }
    }
    tmem_st8(ta_hi + (uint32_t)(g8 * 8), vh);
    if (wlo) tmem_st8(ta_lo + (uint32_t)(g8 * 8), vl);
  }
  tmem_wait_st();
}

constexpr int kVStageBytes = 8 * 2 * kSpec * 8;   // voltages: 8 beams x 2 pols x 32 spectra, cf32

// Output staging.  For Q >= 8 the epilogue collects 8 consecutive windows of every (beam, Stokes
// parameter) row of its lane quadrant in shared memory and then writes each row segment as two
// 16-byte stores (a whole 32-byte sector), instead of scattering 4-byte stores over rows that lie
// megabytes apart.  A quadrant's buffer: 32 beams (16 per M tile) x NS parameters x 8 windows,
// the 16-byte chunks of a beam XOR-swizzled by the beam index; two buffers alternate.
template <int NS, int Q>
struct Stage {
  static constexpr bool kOn = Q >= 8;
  static constexpr int kPeriod = Q >= 8 ? Q / 8 : 1;          // tile pairs per flush
  static constexpr int kRow = NS * 8;                          // floats per beam (0: voltages)
  static constexpr int kBuf = 32 * kRow;                       // floats per quadrant buffer
  static constexpr int kBytes = NS == 0 ? 8 * kVStageBytes       // voltages: 4 KB per epilogue warp
                                        : kOn ? 4 * 2 * kBuf * 4 : 0;   // 4 quadrants x 2 buffers
  __device__ static int index(int jq, int param, int wl) {     // float index within a beam's row
    const int chunk = (param * 2 + (wl >> 2)) ^ (jq & (2 * NS - 1));
    return chunk * 4 + (wl & 3);
  }
};

// kSpecW spectra (32 or 16) of one 32-spectrum tile of an accumulator (pol X at `taddr`, pol Y
// 32 columns on; spectra m0 .. m0 + kSpecW - 1): integrate over windows of Q <= kSpecW spectra and
// store the Stokes parameters, to the staging row `srow` (window wl = w - wbase) or, when staging
// is off, to the output rows at `orow`; every parameter is scaled by `osc` (the squared bandpass
// of the channel when the weights leave it out).
template <int NS, int Q, int kSpecW>
__device__ __forceinline__ void drain_tile(uint32_t taddr, int m0, int ro, int jq, int M, bool beam_ok, float *orow,
                                           long long pstride, float *srow, int wbase, float osc) {
  float x[kSpecW / 16][16], y[kSpecW / 16][16];
#pragma unroll
  for (int ch = 0; ch < kSpecW / 16; ++ch) {
    tmem_ld16(taddr + (uint32_t)(ch * 16), x[ch]);
    tmem_ld16(taddr + (uint32_t)(kSpec + ch * 16), y[ch]);
  }
  tmem_wait_ld();
  // window end: Stokes parameters of the sums, to the staging row or the output rows
  auto window = [&](int ml, float sxx, float syy, float sxy, float sv) {
    const int m = m0 + ml;
    const bool ok = beam_ok && m < M;
    const int w = m / Q;
    if (NS == 1) {
      const float i_own = sxx + syy;
      const float I = osc * (i_own + __shfl_xor_sync(0xffffffffu, i_own, 1));
      if (ok && ro == 0) {
        if (Stage<NS, Q>::kOn) srow[Stage<NS, Q>::index(jq, 0, w - wbase)] = I;
        else orow[w] = I;
      }
    } else {
      // lane ro 0 ends with (I, Q), lane ro 1 with (U, V): each sends what its partner keeps
      const float i_own = sxx + syy, q_own = sxx - syy, u_own = sxy, v_own = ro ? sv : -sv;
      float k0 = ro ? u_own : i_own, k1 = ro ? v_own : q_own;
      const float s0 = ro ? i_own : u_own, s1 = ro ? q_own : v_own;
      k0 += __shfl_xor_sync(0xffffffffu, s0, 1);
      k1 += __shfl_xor_sync(0xffffffffu, s1, 1);
      const float sc = ro ? 2.f * osc : osc;
      k0 *= sc;
      k1 *= sc;
      if (ok) {
        const int p0 = ro ? 2 : 0;
        if (Stage<NS, Q>::kOn) {
          srow[Stage<NS, Q>::index(jq, p0, w - wbase)] = k0;
          srow[Stage<NS, Q>::index(jq, p0 + 1, w - wbase)] = k1;
        } else {
          orow[p0 * pstride + w] = k0;
          orow[(p0 + 1) * pstride + w] = k1;
        }
      }
    }
  };
  if constexpr (Q <= 2) {   // short windows: scalar sums (the pair form spills here)
    float sxx = 0.f, syy = 0.f, sxy = 0.f, sv = 0.f;
#pragma unroll
    for (int ml = 0; ml < kSpecW; ++ml) {
      const float xv = x[ml >> 4][ml & 15], yv = y[ml >> 4][ml & 15];
      sxx = fmaf(xv, xv, sxx);
      syy = fmaf(yv, yv, syy);
      if (NS == 4) {
        sxy = fmaf(xv, yv, sxy);
        sv = fmaf(xv, __shfl_xor_sync(0xffffffffu, yv, 1), sv);   // Im X Re Y (ro 1) or Re X Im Y (ro 0)
      }
      if ((ml + 1) % Q == 0) {
        window(ml, sxx, syy, sxy, sv);
        sxx = syy = sxy = sv = 0.f;
      }
    }
  } else {
    // spectra in pairs: packed FP32x2 FMAs, one per pair and sum (half the instructions and half
    // the dependency chain of scalar sums); the two halves meet at the window's end
    float2 pxx = make_float2(0.f, 0.f), pyy = pxx, pxy = pxx, pv = pxx;
#pragma unroll
    for (int ml = 0; ml < kSpecW; ml += 2) {
      const float2 xv = make_float2(x[ml >> 4][ml & 15], x[ml >> 4][(ml & 15) + 1]);
      const float2 yv = make_float2(y[ml >> 4][ml & 15], y[ml >> 4][(ml & 15) + 1]);
      pxx = __ffma2_rn(xv, xv, pxx);
      pyy = __ffma2_rn(yv, yv, pyy);
      if (NS == 4) {
        pxy = __ffma2_rn(xv, yv, pxy);
        // Im X Re Y (ro 1) or Re X Im Y (ro 0)
        const float2 yp = make_float2(__shfl_xor_sync(0xffffffffu, yv.x, 1), __shfl_xor_sync(0xffffffffu, yv.y, 1));
        pv = __ffma2_rn(xv, yp, pv);
      }
      if ((ml + 2) % Q == 0) {             // a window ends here (compile-time)
        window(ml + 1, pxx.x + pxx.y, pyy.x + pyy.y, pxy.x + pxy.y, pv.x + pv.y);
        pxx = pyy = pxy = pv = make_float2(0.f, 0.f);
      }
    }
  }
}

// One 32-spectrum tile of an accumulator as beam voltages (pol X at `taddr`, pol Y 32 columns on;
// spectra m0 .. m0 + 31) for the 16 beams of this warp's lanes (beam b0 + jq), into vol
// [B][F][N][P][M] cf32 (`vrow0` is the pol-X row of beam b0; rows of one beam are M apart, beams
// `bstride` apart).  The Re lane of a beam keeps the real parts of spectra 0..15 and receives their
// imaginary parts from the Im lane, which keeps the imaginary parts of 16..31 and receives their
// real parts (one shuffle per value).  The complex values then go through the warp's 4 KB of
// shared memory, 8 beams at a time (spectrum index XOR 2 x beam, so the writes hit distinct
// banks), and out as whole 256-byte rows: 16 lanes per (beam, pol) row, two rows per store.
__device__ __forceinline__ void drain_tile_v(uint32_t taddr, int m0, int ro, int jq, int lane, int M, int B, int b0,
                                             float2 *vrow0, long long bstride, bool vec, float2 *stage, float osc) {
  float v[2][2][16];   // [pol][spectrum half][16]
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    tmem_ld16(taddr + (uint32_t)(h * 16), v[0][h]);
    tmem_ld16(taddr + (uint32_t)(kSpec + h * 16), v[1][h]);
  }
  tmem_wait_ld();
  float2 o[2][16];     // this lane's complex values: spectra 16 ro + j, both pols
#pragma unroll
  for (int pol = 0; pol < 2; ++pol)
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const float recv = __shfl_xor_sync(0xffffffffu, ro ? v[pol][0][j] : v[pol][1][j], 1);
      o[pol][j] = ro ? make_float2(recv, v[pol][1][j]) : make_float2(v[pol][0][j], recv);
    }
#pragma unroll
  for (int r = 0; r < 2; ++r) {          // beams 8 r .. 8 r + 7 of the warp's 16
    if ((jq >> 3) == r) {
      const int bl = jq & 7;
#pragma unroll
      for (int pol = 0; pol < 2; ++pol)
#pragma unroll
        for (int j = 0; j < 16; ++j) stage[(bl * 2 + pol) * kSpec + 16 * ro + (j ^ (2 * bl))] = o[pol][j];
    }
    __syncwarp();
    const int j2 = lane & 15;            // spectra 2 j2, 2 j2 + 1 of the row
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int row = 2 * k + (lane >> 4);   // (beam, pol) of the 8 staged beams
      const int bl = row >> 1, pol = row & 1;
      const int b = b0 + 8 * r + bl;
      const int s0 = 2 * j2;                 // spectrum within the tile (even)
      float4 val = *reinterpret_cast<const float4 *>(stage + row * kSpec + (s0 & 16) + ((s0 & 15) ^ (2 * bl)));
      val.x *= osc; val.y *= osc; val.z *= osc; val.w *= osc;
      const int m = m0 + s0;
      if (b < B) {
        float2 *dst = vrow0 + (long long)(8 * r + bl) * bstride + (long long)pol * M + m;
        if (vec && m + 1 < M) {
          *reinterpret_cast<float4 *>(dst) = val;
        } else {
          if (m < M) dst[0] = make_float2(val.x, val.y);
          if (m + 1 < M) dst[1] = make_float2(val.z, val.w);
        }
      }
    }
    __syncwarp();
  }
}

// The rows a thread writes in every flush of a work item (kQT threads per quadrant: thread tq of
// the quadrant's epilogue warps): rows (beam, Stokes parameter) i = tq + kQT k, each written as the
// 16-byte part `part` of a 32-byte segment.  Their addresses depend only on the item, so they are
// formed once per item (null for beams past B, and for threads past the quadrant's 64 NS parts).
template <int NS, int Q>
struct FlushRows {
  static constexpr int kQT = 32 * epi_split<NS, Q>();
  static constexpr int kRowsPer = NS * 2 * 32 / kQT > 0 ? NS * 2 * 32 / kQT : 1;   // rows per thread
  float *row[kRowsPer];
  int soff[kRowsPer];     // float offset of the row's part within the quadrant buffer
  int part;
};

template <int NS, int Q>
__device__ __forceinline__ void flush_rows(const TcParams &p, FlushRows<NS, Q> &fr, int tq, int quad, int bb, int f,
                                           int c) {
  const int Mq = p.M / Q;
  fr.part = tq & 1;
#pragma unroll
  for (int k = 0; k < FlushRows<NS, Q>::kRowsPer; ++k) {
    const int i = tq + FlushRows<NS, Q>::kQT * k;
    const int param = (i >> 1) % NS, bq = (i >> 1) / NS;
    const int jq = bq & 15, mt = bq >> 4;
    const int b = bb * kBeamsPerItem + mt * (kRows / 2) + quad * 16 + jq;
    fr.row[k] = (i < 32 * NS * 2 && b < p.B) ? p.out + ((((long long)b * NS + param) * p.F + f) * kN + c) * Mq
                                              : nullptr;
    fr.soff[k] = bq * Stage<NS, Q>::kRow + ((param * 2 + fr.part) ^ (jq & (2 * NS - 1))) * 4;
  }
}

// Write a quadrant's staged windows wbase .. wbase + 7 to the output rows.
template <int NS, int Q>
__device__ __forceinline__ void flush_stage(const TcParams &p, const float *buf, const FlushRows<NS, Q> &fr,
                                            int wbase) {
  const int Mq = p.M / Q;
  const int w0 = wbase + fr.part * 4;
  if (w0 >= Mq) return;
#pragma unroll
  for (int k = 0; k < FlushRows<NS, Q>::kRowsPer; ++k) {
    if (!fr.row[k]) continue;
    const float4 v = *reinterpret_cast<const float4 *>(buf + fr.soff[k]);
    float *dst = fr.row[k] + w0;
    if (p.vec && w0 + 3 < Mq) {
      *reinterpret_cast<float4 *>(dst) = v;
    } else {
      const float e[4] = {v.x, v.y, v.z, v.w};
      for (int q = 0; q < 4 && w0 + q < Mq; ++q) dst[q] = e[q];
    }
  }
}

// kForm: kMultiPlan (the launch table holds several plans, a batch, each with its own product count)
// or a single plan -- plan 0, its parameters at compile-time offsets into the table -- with three
// (kSingle3) or two (kSingle2) products; a run-time product count costs the single plan ~3 %.
constexpr int kSingle3 = 0, kSingle2 = 1, kMultiPlan = 2;

// TMEM column of the weights of M tile mt: the hi plane (lo = hi + 64 with three products).  The
// single-plan two-product form needs no lo planes, which leaves room for two weight sets used by
// alternate items (set = item parity): the next item's weights are written early in the current
// item, and the MMAs never wait for them at an item boundary.
template <int kForm>
__device__ __forceinline__ uint32_t wcol(int mt, int set) {
  return kForm == kSingle2 ? kACol0 + (uint32_t)(set * 128 + mt * 64) : kACol0 + (uint32_t)(2 * mt * 64);
}
template <int NS, int Q, int kForm>
__global__ void __launch_bounds__(tc_threads<NS, Q>(), 1)
bf_tc_kernel(const __grid_constant__ TcLaunch L) {
  constexpr bool kMulti = kForm == kMultiPlan;
  constexpr int KS = epi_split<NS, Q>();          // epilogue warps per TMEM lane quadrant
  constexpr int kSpecW = 2 * kSpec / KS;          // spectra of a tile one epilogue warp drains
  // whether plan p adds the Wlo Yhi product
  auto wlo_of = [](const TcParams &p) { return kMulti ? p.wlo != 0 : kForm == kSingle3; };
  using St = Stage<NS, Q>;
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char *sbase = smem_raw + (base - raw);
  const uint32_t bar0 = base;
  const uint32_t sB = base + kBarBytes;
  auto full_bar = [&](int s) { return bar0 + 8u * s; };                  // kMaxStages
  auto empty_bar = [&](int s) { return bar0 + 64u + 8u * s; };           // kMaxStages
  auto accf_bar = [&](int mt) { return bar0 + 128u + 8u * mt; };         // accumulator mt committed
  auto acce_bar = [&](int mt) { return bar0 + 144u + 8u * mt; };         // accumulator mt drained
  auto afull_bar = [&](int mt) { return bar0 + 160u + 8u * mt; };        // weights of tile mt written
  auto pair_bar = [&](int q) { return bar0 + 176u + 8u * q; };           // a quadrant's staging filled
  const uint32_t drain_bar = bar0 + 208u;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sbase + 224);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(sbase + 228);
  const int nst = L.nstages;
  float *const stage_out = reinterpret_cast<float *>(sbase + kBarBytes + (size_t)nst * L.stage_max);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int mt = 0; mt < kMTiles; ++mt) {
      mbar_init(accf_bar(mt), 1);
      mbar_init(acce_bar(mt), 4 * KS);     // one arrival per epilogue warp
      mbar_init(afull_bar(mt), 4 * KS);
    }
    for (int q = 0; q < 4; ++q) mbar_init(pair_bar(q), KS);
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      int s = 0, issued_n = 0;           // ring stage and the number of stages filled so far
      uint32_t ph = 0;                   // phase parity of stage s
      bool ok = true, stalled = false;
      for (int item = blockIdx.x; item < L.items && ok; item += gridDim.x) {
        if ((long long)item == L.stall_item) { stalled = true; break; }   // test hook: a barrier nothing fills
        const int pi = kMulti ? plan_of(L, item) : 0;
        const TcParams &p = L.plan[pi];
        const int fc = (item - p.first_item) / p.items_per_fc;
        const uint32_t bytes = (uint32_t)p.stage_bytes;
        const uint32_t plane_bytes = bytes / 2;    // two tiles of one plane
        for (int t = 0; t < p.ntiles; ++t) {
          if (!mbar_wait(empty_bar(s), ph ^ 1u, abort_flag)) { fail(abort_flag, p.err, ERR_PRODUCER); ok = false; break; }
          mbar_expect_tx(full_bar(s), bytes);
          const uint32_t dst = sB + (uint32_t)s * (uint32_t)L.stage_max;
          tma_load_4d(dst, &L.map[2 * pi], 0, 0, 2 * t, fc, full_bar(s));
          tma_load_4d(dst + plane_bytes, &L.map[2 * pi + 1], 0, 0, 2 * t, fc, full_bar(s));
          ++issued_n;
          if (++s == nst) { s = 0; ph ^= 1u; }
        }
      }
      if (*abort_flag || stalled) {   // let our own copies land before the shared memory goes away
        // the last min(issued, nst) fills, newest first: stage s - 1, s - 2, ... (wrapping)
        int q = s;
        uint32_t qph = ph;
        for (int k = 0; k < nst && k < issued_n; ++k) {
          if (q == 0) { q = nst; qph ^= 1u; }
          --q;
          volatile int never = 0;
          mbar_wait(full_bar(q), qph, &never);
        }
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      bool issued = false, ok = true;
      int s = 0, it = 0;
      uint32_t ph = 0, gpar = 0;         // ring stage and its phase parity; tile-pair parity
      int *err = L.plan[0].err;
      for (int item = blockIdx.x; item < L.items && ok; item += gridDim.x, ++it) {
        const TcParams &p = L.plan[kMulti ? plan_of(L, item) : 0];
        err = p.err;
        const int ksteps = p.Kpad >> 4;
        const bool wlo = wlo_of(p);     // read once: the MMA asm clobbers memory
        const uint32_t plane_bytes = (uint32_t)p.stage_bytes / 2;
        const uint64_t desc_b0 = smem_desc(sB, (uint32_t)(p.Kpad * 128));   // stage 0, hi plane, k step 0
        for (int t = 0; t < p.ntiles && ok; ++t, gpar ^= 1u) {
          if (!mbar_wait(full_bar(s), ph, abort_flag)) { fail(abort_flag, p.err, ERR_MMA); ok = false; break; }
          for (int mt = 0; mt < kMTiles; ++mt) {
            if (t == 0 && !mbar_wait(afull_bar(mt), (uint32_t)it & 1u, abort_flag)) {
              fail(abort_flag, p.err, ERR_MMA); ok = false; break;
            }
            if (!mbar_wait(acce_bar(mt), gpar ^ 1u, abort_flag)) {
              fail(abort_flag, p.err, ERR_MMA); ok = false; break;
            }
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)(mt * kAccCols);
            uint32_t a_hi = tmem + wcol<kForm>(mt, it & 1);
            // descriptors advance by adding the byte offset / 16 to the start-address field (all
            // shared addresses are below 256 KB, so the 14-bit field never carries)
            uint64_t b_hi = desc_b0 + (uint64_t)((s * L.stage_max) >> 4);
            for (int ks = 0; ks < ksteps; ++ks) {
              const uint64_t b_lo = b_hi + (uint64_t)(plane_bytes >> 4);
              umma(d, a_hi, b_hi, ks != 0);           // Whi Yhi
              if (wlo) umma(d, a_hi + 64u, b_hi, 1);     // Wlo Yhi
              umma(d, a_hi, b_lo, 1);                 // Whi Ylo
              a_hi += 8u;                             // 16 K elements = 8 TMEM columns
              b_hi += (uint64_t)((16 * 128) >> 4);    // 16 K rows of 128 bytes
            }
            umma_commit(accf_bar(mt));
            issued = true;
          }
          if (ok) umma_commit(empty_bar(s));
          if (++s == nst) { s = 0; ph ^= 1u; }
        }
      }
      if (issued) {   // every MMA (and its barrier arrivals) retired before TMEM is released
        umma_commit(drain_bar);
        volatile int never = 0;
        if (!mbar_wait(drain_bar, 0, &never)) fail(abort_flag, err, ERR_MMA);
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogue: weights, TMEM -> Stokes
    // warp (quad, half): TMEM lanes 32 quad .. +31 of both M tiles; weight columns of groups
    // g8 = half (mod KS); of every tile pair t, spectra q2 kSpecW .. + kSpecW - 1 of tile 2t + h
    const int quad = warp & 3, half = (warp - 2) >> 2;
    const int h = half / (KS / 2), q2 = half % (KS / 2);
    const int ro = lane & 1;              // 0: Re V rows, 1: Im V rows
    const int jq = lane >> 1;             // beam within the quadrant (16 per M tile)
    const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
    float *const qbuf = stage_out + quad * 2 * St::kBuf;
    uint32_t gpar = 0;                   // tile-pair parity
    int fl = 0, eit = 0;                 // staging flushes; items of this CTA so far
    bool ok = true;
    constexpr bool kTwoSets = kForm == kSingle2;
    for (int item = blockIdx.x; item < L.items && ok; item += gridDim.x, ++eit) {
      const TcParams &p = L.plan[kMulti ? plan_of(L, item) : 0];
      const int Mq = p.M / Q;
      const long long pstride = (long long)p.F * kN * Mq;      // between Stokes parameters
      const int li = item - p.first_item;
      const int fc = li / p.items_per_fc;
      const int bb = li - fc * p.items_per_fc;
      const int f = fc / kN, c = fc - f * kN;
      // bandpass of the channel when the planes precede it (applied to the outputs: the weights
      // stay unit phasors, whose FP16 rounding is finest below 1)
      const float bpc = p.bp ? __ldg(&p.bp[c]) : 1.f;
      if (item == (int)blockIdx.x) {      // weights of the first item; later ones are written during the
        for (int mt = 0; mt < kMTiles; ++mt) {   // item before (its first or last tile pair)
          const uint32_t ta_hi = tmem + lane_off + wcol<kForm>(mt, 0);
          WeightTables<KS> tab;
          load_weight_tables(p, f, bb * kBeamsPerItem + mt * (kRows / 2) + quad * 16 + jq, ro, half, tab);
          write_weights(p, ta_hi, ta_hi + 64u, c, ro, half, tab, wlo_of(p));
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(afull_bar(mt));
        }
      }
      // the next item of this CTA (possibly of another plan): its weights follow this item's last tile
      const int nitem = item + gridDim.x;
      const TcParams &pn = L.plan[kMulti ? plan_of(L, nitem < L.items ? nitem : item) : 0];
      const int nli = nitem - pn.first_item;
      const int nfc = nli / pn.items_per_fc;
      const int nbb = nli - nfc * pn.items_per_fc;
      FlushRows<NS, Q> frows;
      if constexpr (St::kOn) flush_rows<NS, Q>(p, frows, half * 32 + lane, quad, bb, f, c);   // tq
      for (int t = 0; t < p.ntiles && ok; ++t, gpar ^= 1u) {
        const int wbase = (t / St::kPeriod) * 8;
        float *const buf = qbuf + (fl & 1) * St::kBuf;
        for (int mt = 0; mt < kMTiles; ++mt) {
          // write the next item's weights after this tile pair: with one weight set, after the
          // last (the MMAs reading this tile's weights are then complete); with two, after the
          // first (the other set's last reader, the previous item, is then complete)
          const bool boundary = (kTwoSets ? t == 0 : t == p.ntiles - 1) && nitem < L.items;
          WeightTables<KS> tab;
          if (boundary)   // the next item's table values, in flight while the last accumulator fills
            load_weight_tables(pn, nfc / kN, nbb * kBeamsPerItem + mt * (kRows / 2) + quad * 16 + jq, ro, half, tab);
          if (!mbar_wait(accf_bar(mt), gpar, abort_flag)) { fail(abort_flag, p.err, ERR_EPILOGUE); ok = false; break; }
          tc_fence_after();
          const int b = bb * kBeamsPerItem + mt * (kRows / 2) + quad * 16 + jq;
          const uint32_t taddr = tmem + lane_off + (uint32_t)(mt * kAccCols + h * 2 * kSpec + q2 * kSpecW);
          const int m0 = t * 2 * kSpec + h * kSpec + q2 * kSpecW;
          if constexpr (NS == 0) {
            const int b0 = bb * kBeamsPerItem + mt * (kRows / 2) + quad * 16;   // beam of lanes 0, 1
            const long long bstride = (long long)p.F * kN * kP * p.M;             // between beams
            float2 *const v0 = reinterpret_cast<float2 *>(p.out) + (((long long)b0 * p.F + f) * kN + c) * kP * p.M;
            drain_tile_v(taddr, m0, ro, jq, lane, p.M, p.B, b0, v0, bstride, p.vec != 0,
                         reinterpret_cast<float2 *>(stage_out) + (warp - 2) * (kVStageBytes / 8), bpc);
          } else {
            float *const orow = p.out + (((long long)b * NS * p.F + f) * kN + c) * Mq;
            drain_tile<NS, Q, kSpecW>(taddr, m0, ro, jq, p.M, b < p.B, orow, pstride, buf + (mt * 16 + jq) * St::kRow,
                                      wbase, bpc * bpc);
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(acce_bar(mt));
          if (boundary) {
            const uint32_t ta_hi = tmem + lane_off + wcol<kForm>(mt, (eit + 1) & 1);
            write_weights(pn, ta_hi, ta_hi + 64u, nfc % kN, ro, half, tab, wlo_of(pn));
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(afull_bar(mt));
          }
        }
        if constexpr (St::kOn) {
        if (ok && ((t + 1) % St::kPeriod == 0 || t == p.ntiles - 1)) {
          // both warps of the quadrant have staged their windows: write the rows out
          __syncwarp();
          if (lane == 0) mbar_arrive(pair_bar(quad));
          if (!mbar_wait(pair_bar(quad), (uint32_t)fl & 1u, abort_flag)) { fail(abort_flag, p.err, ERR_EPILOGUE); ok = false; break; }
          flush_stage<NS, Q>(p, buf, frows, wbase);
          ++fl;
        }
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

template <int NS, int Q, int kForm>
cudaError_t launch_q(TcLaunch &L, int grid, cudaStream_t st) {
  // B ring: as many stages of the largest plan as shared memory leaves after the barriers and
  // the output staging
  L.nstages = (kRingBytes - Stage<NS, Q>::kBytes) / L.stage_max;
  if (L.nstages > kMaxStages) L.nstages = kMaxStages;
  if (L.nstages < 2) return cudaErrorInvalidValue;
  int smem = 1024 + kBarBytes + L.nstages * L.stage_max + Stage<NS, Q>::kBytes;
  // at least half of an SM's shared memory, so that no two CTAs share an SM (each holds all of
  // its TMEM columns)
  if (smem < kMinSmem) smem = kMinSmem;
  cudaError_t e = cudaFuncSetAttribute(bf_tc_kernel<NS, Q, kForm>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  bf_tc_kernel<NS, Q, kForm><<<grid, tc_threads<NS, Q>(), smem, st>>>(L);
  return cudaGetLastError();
}

template <int NS, int kForm>
cudaError_t launch_ns(int Q, TcLaunch &L, int grid, cudaStream_t st) {
  switch (Q) {
    case 1: return launch_q<NS, 1, kForm>(L, grid, st);
    case 2: return launch_q<NS, 2, kForm>(L, grid, st);
    case 4: return launch_q<NS, 4, kForm>(L, grid, st);
    case 8: return launch_q<NS, 8, kForm>(L, grid, st);
    case 16: return launch_q<NS, 16, kForm>(L, grid, st);
    case 32: return launch_q<NS, 32, kForm>(L, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

int sm_count() {
  static int n[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  if (!n[dev] && cudaDeviceGetAttribute(&n[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) n[dev] = 0;
  return n[dev];
}

// Plan i of a launch: its parameters from the geometry, its work items after the previous plans'.
bool fill_plan(TcLaunch &L, int i, const Geometry &g, int out_kind, const void *tm_hi, const void *tm_lo, float *out,
               int *err) {
  if (!tm_hi || !tm_lo || g.S > tc_max_stations()) return false;
  TcParams &p = L.plan[i];
  p.S = g.S; p.F = g.F; p.B = g.B; p.M = g.M;
  p.Kpad = tc_kpad(g.S);
  p.stage_bytes = 4 * p.Kpad * 128;
  p.ntiles = tc_tiles(g.M) / 2;
  p.items_per_fc = (g.B + kBeamsPerItem - 1) / kBeamsPerItem;
  const long long items = (long long)g.F * kN * p.items_per_fc;
  const long long first = i == 0 ? 0 : (long long)L.plan[i - 1].first_item + L.plan[i - 1].items;
  if (items + first >= (1ll << 31)) return false;
  p.items = (int)items;
  p.first_item = (int)first;
  // raw planes (the fused path): weights with the delay compensation folded in, outputs scaled by
  // the bandpass
  p.phase0 = g.ct16_raw ? g.phase0g : g.phase0;
  p.step = g.ct16_raw ? g.stepg : g.step;
  p.bp = g.ct16_raw ? g.bandpass : nullptr;
  if (!p.phase0 || !p.step) return false;
  p.out = out; p.err = err;
  p.wlo = g.tc_wlo ? 1 : 0;
  const bool aligned = (reinterpret_cast<uintptr_t>(out) & 15) == 0;
  p.vec = out_kind == OUT_VOLTAGES ? (g.M % 2 == 0 && aligned) : ((g.M / g.Q) % 4 == 0 && aligned);
  L.map[2 * i] = *reinterpret_cast<const CUtensorMap *>(tm_hi);
  L.map[2 * i + 1] = *reinterpret_cast<const CUtensorMap *>(tm_lo);
  L.items = p.first_item + p.items;
  L.stage_max = p.stage_bytes > L.stage_max ? p.stage_bytes : L.stage_max;
  L.nplans = i + 1;
  return true;
}

template <int kForm>
cudaError_t launch_form(TcLaunch &L, int out_kind, int Q, int grid, cudaStream_t st) {
  if (out_kind == OUT_VOLTAGES) return launch_q<0, 1, kForm>(L, grid, st);
  if (out_kind == OUT_STOKES_IQUV) return launch_ns<4, kForm>(Q, L, grid, st);
  if (out_kind == OUT_STOKES_I) return launch_ns<1, kForm>(Q, L, grid, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_table(TcLaunch &L, int out_kind, int Q, cudaStream_t st) {
  if (L.items == 0) return cudaSuccess;
  const int sms = sm_count();
  if (sms <= 0) return cudaErrorInvalidDevice;
  const int grid = L.items < sms ? L.items : sms;
  if (L.nplans > 1) return launch_form<kMultiPlan>(L, out_kind, Q, grid, st);
  return L.plan[0].wlo ? launch_form<kSingle3>(L, out_kind, Q, grid, st)
                       : launch_form<kSingle2>(L, out_kind, Q, grid, st);
}

}  // namespace

int tc_max_stations() { return kMaxKpad / 2; }
int tc_spectra_per_tile() { return kSpec; }
int tc_kpad(int S) { return ((2 * S + 15) / 16) * 16; }
int tc_max_plans_per_launch() { return kMaxPlans; }

cudaError_t launch_bf_tc(const Geometry &g, int out_kind, const void *tm_hi, const void *tm_lo, float *out, int *err,
                         cudaStream_t st, long long stall_item) {
  if (g.M == 0 || g.B == 0) return cudaSuccess;
  TcLaunch L;
  L.nplans = 0; L.items = 0; L.nstages = 0; L.stage_max = 0;
  L.stall_item = stall_item;
  if (!fill_plan(L, 0, g, out_kind, tm_hi, tm_lo, out, err)) return cudaErrorInvalidValue;
  return launch_table(L, out_kind, g.Q, st);
}

cudaError_t launch_bf_tc_group(const TcPlanRef *plans, int n, int out_kind, int Q, cudaStream_t st) {
  if (n < 1 || n > kMaxPlans) return cudaErrorInvalidValue;
  TcLaunch L;
  L.nplans = 0; L.items = 0; L.nstages = 0; L.stage_max = 0;
  L.stall_item = -1;
  int k = 0;
  for (int i = 0; i < n; ++i) {
    const TcPlanRef &r = plans[i];
    if (r.g.Q != Q && out_kind != OUT_VOLTAGES) return cudaErrorInvalidValue;
    if (r.g.M == 0 || r.g.B == 0) continue;
    if (!fill_plan(L, k, r.g, out_kind, r.tm_hi, r.tm_lo, r.out, r.err)) return cudaErrorInvalidValue;
    ++k;
  }
  return launch_table(L, out_kind, Q, st);
}

}  // namespace lbf
