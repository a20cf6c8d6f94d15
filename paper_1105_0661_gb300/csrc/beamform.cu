// Tied-array beam former (Section 4.3) with on-the-fly positional weights and an optional fused
// Stokes / time-integration epilogue (Sections 4.5, 5.1).
//
// Per (subband f, channel c) the work is a complex product  V[b][pol, m] = sum_s w[b,s] Y[s][pol, m]
// with w[b,s] = exp(+2 pi i f_c dtau[b,s]), f_c = f0_f + df_c.  The weights are generated per CTA
// into shared memory from the plan's FP64-reduced phase tables (tables.cu) and an FP32 sincos.
//
// Two kernels:
//  * few-beam (bandwidth bound): one thread per spectrum m (both pols), weights broadcast from
//    shared memory, one coalesced pass over the corner-turned input; Stokes integration over Q
//    consecutive spectra is a warp-shuffle reduction across the lanes that hold them.
//  * many-beam (FP32-ALU bound): 128 beams x 32 spectra per CTA pass, each thread a 4-beam x
//    4-spectrum x 2-pol register tile (32 complex accumulators); the corner-turned input passes
//    are double-buffered in shared memory by cp.async, and every station step issues 128 FFMAs
//    per 6 conflict-free shared-memory vector loads.
#include "lbf_internal.cuh"

namespace lbf {
namespace {

constexpr int kFewThreads = 256;
constexpr int kFewBeams = 8;     // beams per few-beam CTA (grid.y covers more; 16 for some B)
constexpr int kManyThreads = 256;
constexpr int kBT = 128;         // beams per many-beam CTA
constexpr int kMC = 32;          // spectra per many-beam pass

__device__ __forceinline__ void cmac(float2 &acc, float2 w, float2 y) {
  acc.x = fmaf(w.x, y.x, acc.x);
  acc.x = fmaf(-w.y, y.y, acc.x);
  acc.y = fmaf(w.x, y.y, acc.y);
  acc.y = fmaf(w.y, y.x, acc.y);
}

// Stokes parameter `st` of the voltage pair (X, Y), Section 4.5.
__device__ __forceinline__ float stokes_param(int st, float2 X, float2 Y) {
  const float xx = fmaf(X.x, X.x, X.y * X.y);
  const float yy = fmaf(Y.x, Y.x, Y.y * Y.y);
  switch (st) {
    case 0: return xx + yy;                                   // I
    case 1: return xx - yy;                                   // Q
    case 2: return 2.f * fmaf(X.x, Y.x, X.y * Y.y);           // U = 2 Re(X conj Y)
    default: return 2.f * fmaf(X.y, Y.x, -X.x * Y.y);         // V = 2 Im(X conj Y)
  }
}

// Incoherent beam (Section 3): the Stokes parameters of the unweighted station signals, summed
// over stations as powers -- accumulated per spectrum as sum |X|^2, sum |Y|^2 and sum X conj Y.
struct IncAcc {
  float xx = 0.f, yy = 0.f, re = 0.f, im = 0.f;
  __device__ __forceinline__ void add(float2 X, float2 Y) {
    xx = fmaf(X.x, X.x, fmaf(X.y, X.y, xx));
    yy = fmaf(Y.x, Y.x, fmaf(Y.y, Y.y, yy));
    re = fmaf(X.x, Y.x, fmaf(X.y, Y.y, re));
    im = fmaf(X.y, Y.x, fmaf(-X.x, Y.y, im));
  }
  __device__ __forceinline__ float param(int st) const {
    switch (st) {
      case 0: return xx + yy;
      case 1: return xx - yy;
      case 2: return 2.f * re;
      default: return 2.f * im;
    }
  }
};

// ------------------------------------------------------------------------------- few beams
// Work item: (subband, channel) fc, beams bgrp * FB .. + FB - 1.  FB = 16 reads the corner-turned
// block half as often for 9 to 32 beams (16 FP32 flop per byte, about the FP32/HBM ridge).
template <int OUT, int FB = kFewBeams>
__device__ __forceinline__ void bf_few_item(const Geometry &g, const float2 *__restrict__ ct, void *__restrict__ out,
                                            int fc, int bgrp, float2 *wsm /* [S][FB] */) {
  const int f = fc / kN, c = fc - f * kN;
  const int b0 = bgrp * FB;
  const int tid = threadIdx.x;
  for (int i = tid; i < g.S * FB; i += kFewThreads) {
    const int s = i / FB, b = b0 + (i - s * FB);
    wsm[i] = (b < g.B) ? beam_weight(g, f, c, (long long)b * g.S + s) : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const float2 *y = ct + (long long)fc * g.S * kP * g.M;
  const int nS = (OUT == OUT_STOKES_IQUV) ? 4 : 1;
  const int Mq = g.M / g.Q;
  for (int mb = 0; mb < g.M; mb += kFewThreads) {
    const int m = mb + tid;
    const bool active = m < g.M;
    float2 acc[FB][kP];
#pragma unroll
    for (int b = 0; b < FB; ++b) acc[b][0] = acc[b][1] = make_float2(0.f, 0.f);
    const bool inc = OUT != OUT_VOLTAGES && g.inc && bgrp == 0;   // this item also forms beam B
    IncAcc ia;
    if (active) {
      // unrolled so that the loads of several stations are in flight together (the kernel is
      // bound by HBM latency x loads in flight, not by its arithmetic)
#pragma unroll 4
      for (int s = 0; s < g.S; ++s) {
        const float2 yx = y[((long long)s * kP + 0) * g.M + m];
        const float2 yy = y[((long long)s * kP + 1) * g.M + m];
        if (inc) ia.add(yx, yy);
        const float4 *w4 = reinterpret_cast<const float4 *>(wsm + s * FB);
#pragma unroll
        for (int b2 = 0; b2 < FB / 2; ++b2) {
          const float4 w = w4[b2];
          cmac(acc[2 * b2][0], make_float2(w.x, w.y), yx);
          cmac(acc[2 * b2][1], make_float2(w.x, w.y), yy);
          cmac(acc[2 * b2 + 1][0], make_float2(w.z, w.w), yx);
          cmac(acc[2 * b2 + 1][1], make_float2(w.z, w.w), yy);
        }
      }
    }
    if (OUT == OUT_VOLTAGES) {
      if (active) {
        float2 *vol = reinterpret_cast<float2 *>(out);
#pragma unroll
        for (int b = 0; b < FB; ++b)
          if (b0 + b < g.B)
#pragma unroll
            for (int pol = 0; pol < kP; ++pol)
              vol[((((long long)(b0 + b) * g.F + f) * kN + c) * kP + pol) * g.M + m] = acc[b][pol];
      }
    } else {
      float *o = reinterpret_cast<float *>(out);
#pragma unroll
      for (int b = 0; b < FB; ++b) {
        if (b0 + b >= g.B) break;   // uniform across the CTA
#pragma unroll
        for (int st = 0; st < nS; ++st) {
          float v = stokes_param(st, acc[b][0], acc[b][1]);
          for (int o2 = 1; o2 < g.Q; o2 <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o2);
          if (active && (m & (g.Q - 1)) == 0)
            o[((((long long)(b0 + b) * nS + st) * g.F + f) * kN + c) * Mq + m / g.Q] = v;
        }
      }
      if (inc) {
#pragma unroll
        for (int st = 0; st < nS; ++st) {
          float v = ia.param(st);
          for (int o2 = 1; o2 < g.Q; o2 <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o2);
          if (active && (m & (g.Q - 1)) == 0)
            o[((((long long)g.B * nS + st) * g.F + f) * kN + c) * Mq + m / g.Q] = v;
        }
      }
    }
  }
  __syncthreads();   // the weights in shared memory are rewritten by the next work item
}

// at least two CTAs per SM (three for the 8-beam Stokes I form): a bandwidth-bound kernel needs
// the warps; left to itself the compiler gave the IQUV form 194 registers, one CTA per SM and 2.6x
// the Stokes I time
template <int OUT, int FB>
__global__ void __launch_bounds__(kFewThreads, (OUT == OUT_STOKES_I && FB == 8) ? 3 : 2)
bf_few_kernel(Geometry g, const float2 *__restrict__ ct, void *__restrict__ out) {
  extern __shared__ __align__(16) float2 wsm[];
  bf_few_item<OUT, FB>(g, ct, out, blockIdx.x, blockIdx.y, wsm);
}

template <int FB>
cudaError_t launch_few(const Geometry &g, int out_kind, const float2 *ct, void *out, cudaStream_t st) {
  dim3 grid((unsigned)(g.F * kN), (unsigned)((g.B + FB - 1) / FB));
  const size_t smem = (size_t)g.S * FB * sizeof(float2);
  auto go = [&](auto kern) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kFewThreads, smem, st>>>(g, ct, out);
    return cudaGetLastError();
  };
  switch (out_kind) {
    case OUT_VOLTAGES: return go(bf_few_kernel<OUT_VOLTAGES, 8>);
    case OUT_STOKES_I: return go(bf_few_kernel<OUT_STOKES_I, FB>);
    default: return go(bf_few_kernel<OUT_STOKES_IQUV, 8>);
  }
}

// ------------------------------------------------------------------------------- many beams
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src, int src_bytes) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(gmem_src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gmem_src, int src_bytes) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(gmem_src), "r"(src_bytes) : "memory");
}

// Two tile shapes, both 256 threads and 32-spectrum passes:
//  * BT = 128 beams per CTA: thread tile beams 4 bg .. 4 bg + 3 (bg = tid / 8), spectra {2 mg,
//    2 mg + 1, 16 + 2 mg, 17 + 2 mg} (mg = tid % 8) of the pass, both pols: 32 complex
//    accumulators, 6 16-byte shared loads per station for 128 FFMAs;
//  * BT = 64 beams per CTA: beams 4 bg .. +3 (bg = tid / 16), spectra {2 mg, 2 mg + 1}
//    (mg = tid % 16): 16 complex accumulators, 4 loads per 64 FFMAs, a third of the shared memory
//    per CTA (three CTAs per SM).  A plan whose beam count leaves most of a 128-beam tile empty
//    (24, 154 or 269 beams) wastes less work in 64-beam tiles.
// Each 16-byte shared load of a warp covers 128 contiguous bytes.  Four scalar FMAs per complex
// multiply-add.  The station loop is not unrolled, walks two pointers, and has the beams
// innermost: measured on the LOFAR block, this lowers the FP32 pipe's dispatch stalls (11 %
// faster than unrolling by 2 with the spectra innermost), as does the planar weight layout
// (another 4 %).
// Work item: (subband, channel) fc, beams bt * BT .. + BT - 1.
template <int OUT, int BT>
__device__ __forceinline__ void bf_many_item(const Geometry &g, const float2 *__restrict__ ct, void *__restrict__ out,
                                             int fc, int bt, float2 *smem) {
  constexpr int kJ = BT == 128 ? 4 : 2;   // spectra per thread in a pass
  constexpr int kLanesM = kMC / kJ;       // threads sharing a beam group (8 or 16)
  float2 *wsm = smem;                     // [S][BT / 4][re x4, im x4]
  float2 *ysm = smem + (size_t)g.S * BT;  // [2 buffers][S][kP][kMC]
  const int tid = threadIdx.x;
  const int f = fc / kN, c = fc - f * kN;
  const int bbase = bt * BT;
  const float2 *y = ct + (long long)fc * g.S * kP * g.M;
  const int rows = g.S * kP;
  const size_t ybuf = (size_t)rows * kMC;
  const bool even_m = (g.M & 1) == 0;

  // async copy of pass `mc` into buffer `bi` (zero-filled beyond M)
  auto load_pass = [&](int mc, int bi) {
    float2 *dst = ysm + bi * ybuf;
    if (even_m) {
      for (int i = tid; i < rows * (kMC / 2); i += kManyThreads) {
        const int row = i / (kMC / 2), col = 2 * (i - row * (kMC / 2));
        const int m = mc + col;
        const int valid = m < g.M ? 16 : 0;
        cp_async16(dst + row * kMC + col, y + (long long)row * g.M + (valid ? m : 0), valid);
      }
    } else {
      for (int i = tid; i < rows * kMC; i += kManyThreads) {
        const int row = i / kMC, col = i - row * kMC;
        const int m = mc + col;
        const int valid = m < g.M ? 8 : 0;
        cp_async8(dst + row * kMC + col, y + (long long)row * g.M + (valid ? m : 0), valid);
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  load_pass(0, 0);

  // weights of each group of four beams stored planar: re[4] then im[4], so that a beam's real
  // and imaginary parts land in registers of the same parity (see the inner loop)
  for (int i = tid; i < g.S * BT; i += kManyThreads) {
    const int s = i / BT, bl = i - s * BT, b = bbase + bl;
    const float2 w = (b < g.B) ? beam_weight(g, f, c, (long long)b * g.S + s) : make_float2(0.f, 0.f);
    float *wg = reinterpret_cast<float *>(wsm + s * BT + (bl & ~3));
    wg[bl & 3] = w.x;
    wg[4 + (bl & 3)] = w.y;
  }
  const int bg = tid / kLanesM;   // beams bbase + 4 bg .. +3
  const int mg = tid % kLanesM;   // spectra 2 mg, 2 mg + 1 (and 16 + 2 mg, 17 + 2 mg for BT = 128)
  // spectrum of accumulator jm within the pass
  auto mof = [&](int jm) { return 16 * (jm >> 1) + 2 * mg + (jm & 1); };
  const int nS = (OUT == OUT_STOKES_IQUV) ? 4 : 1;
  const int Mq = (OUT == OUT_VOLTAGES) ? 0 : g.M / g.Q;

  int buf = 0;
  for (int mc = 0; mc < g.M; mc += kMC, buf ^= 1) {
    if (mc + kMC < g.M) load_pass(mc + kMC, buf ^ 1);
    else asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    __syncthreads();   // pass mc (and the weights) visible to every thread
    const float2 *yb = ysm + buf * ybuf;
    if (OUT != OUT_VOLTAGES && g.inc && bt == 0 && tid < kMC) {   // warp 0: incoherent beam B
      IncAcc ia;
      for (int s = 0; s < g.S; ++s) ia.add(yb[(s * kP + 0) * kMC + tid], yb[(s * kP + 1) * kMC + tid]);
      float *o = reinterpret_cast<float *>(out);
      const int m = mc + tid;
      for (int st = 0; st < nS; ++st) {
        float v = ia.param(st);
        for (int o2 = 1; o2 < g.Q; o2 <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o2);
        if (m < g.M && (m & (g.Q - 1)) == 0)
          o[((((long long)g.B * nS + st) * g.F + f) * kN + c) * Mq + m / g.Q] = v;
      }
    }

    float2 acc[4][kP][kJ];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int pol = 0; pol < kP; ++pol)
#pragma unroll
        for (int jm = 0; jm < kJ; ++jm) acc[i][pol][jm] = make_float2(0.f, 0.f);

    const float4 *wp = reinterpret_cast<const float4 *>(wsm + bg * 4);
    const float4 *yp = reinterpret_cast<const float4 *>(yb + 2 * mg);
#pragma unroll 1
    for (int s = 0; s < g.S; ++s, wp += BT / 2, yp += kP * kMC / 2) {
      const float4 wre = wp[0], wim = wp[1];
      const float2 w[4] = {make_float2(wre.x, wim.x), make_float2(wre.y, wim.y),
                           make_float2(wre.z, wim.z), make_float2(wre.w, wim.w)};
#pragma unroll
      for (int pol = 0; pol < kP; ++pol) {
        float2 yv[kJ];
        const float4 ya = yp[pol * (kMC / 2)];
        yv[0] = make_float2(ya.x, ya.y);
        yv[1] = make_float2(ya.z, ya.w);
        if constexpr (kJ == 4) {
          const float4 yc = yp[pol * (kMC / 2) + 8];
          yv[2] = make_float2(yc.x, yc.y);
          yv[3] = make_float2(yc.z, yc.w);
        }
#pragma unroll
        for (int jm = 0; jm < kJ; ++jm)
#pragma unroll
          for (int i = 0; i < 4; ++i) cmac(acc[i][pol][jm], w[i], yv[jm]);
      }
    }

    if (OUT == OUT_VOLTAGES) {
      float2 *vol = reinterpret_cast<float2 *>(out);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int b = bbase + bg * 4 + i;
        if (b >= g.B) continue;
#pragma unroll
        for (int pol = 0; pol < kP; ++pol)
#pragma unroll
          for (int jm = 0; jm < kJ; ++jm) {
            const int m = mc + mof(jm);
            if (m < g.M) vol[((((long long)b * g.F + f) * kN + c) * kP + pol) * g.M + m] = acc[i][pol][jm];
          }
      }
    } else {
      float *o = reinterpret_cast<float *>(out);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int b = bbase + bg * 4 + i;
#pragma unroll
        for (int st = 0; st < nS; ++st) {
          float v[kJ];
#pragma unroll
          for (int jm = 0; jm < kJ; ++jm) v[jm] = stokes_param(st, acc[i][0][jm], acc[i][1][jm]);
          float *orow = o + ((((long long)b * nS + st) * g.F + f) * kN + c) * Mq;
          if (g.Q == 1) {
#pragma unroll
            for (int jm = 0; jm < kJ; ++jm) {
              const int m = mc + mof(jm);
              if (b < g.B && m < g.M) orow[m] = v[jm];
            }
          } else if (kJ == 4 && g.Q == 32) {
            float sum = (v[0] + v[1]) + (v[kJ - 2] + v[kJ - 1]);
            for (int o2 = 1; o2 < kLanesM; o2 <<= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o2);
            if (b < g.B && mg == 0 && mc < g.M) orow[mc / 32] = sum;
          } else {
            // windows of Q consecutive spectra: pair sums, then across the Q/2 lanes of mg that
            // hold the window's other pairs (BT = 64: all 32 spectra of the pass are in one run
            // of 16 lanes, so Q = 32 is this case too)
#pragma unroll
            for (int h = 0; h < kJ / 2; ++h) {
              float sum = v[2 * h] + v[2 * h + 1];
#pragma unroll
              for (int o2 = 1; o2 < kLanesM; o2 <<= 1)
                if (o2 < g.Q / 2) sum += __shfl_xor_sync(0xffffffffu, sum, o2);
              const int m = mc + 16 * h + 2 * mg;
              if (b < g.B && m < g.M && (mg & (g.Q / 2 - 1)) == 0) orow[m / g.Q] = sum;
            }
          }
        }
      }
    }
    __syncthreads();   // everyone is done with buffer `buf` before it is refilled
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// Three 64-beam CTAs per SM fit the shared memory; the IQUV epilogue needs more than the 85
// registers per thread that three CTAs leave, so that form runs two.
template <int OUT, int BT>
__global__ void __launch_bounds__(kManyThreads, (BT == 128 || OUT == OUT_STOKES_IQUV) ? 2 : 3)
bf_many_kernel(Geometry g, const float2 *__restrict__ ct, void *__restrict__ out, int nbt) {
  extern __shared__ __align__(16) float2 smem[];
  const int fc = blockIdx.x / nbt;
  bf_many_item<OUT, BT>(g, ct, out, fc, blockIdx.x - fc * nbt, smem);
}

// Persistent beam former over the blocks of several observations (a batch): CTAs take work items
// (subband-channel, beam group) from a shared counter; each item runs the body of variant V (1 few,
// 2 many with 128-beam tiles, 3 many with 64-beam tiles) for output kind OUT.  One launch per
// (variant, output kind, residency) class, so that each body keeps its own registers and shared
// memory footprint, as when its observation runs alone.  The observations' geometry comes in a
// grid-constant table (constant bank); thread 0 finds each item's observation.
template <int V, int OUT>
__global__ void __launch_bounds__(kManyThreads, (V == 3 && OUT != OUT_STOKES_IQUV) ? 3 : 2)
bf_group_kernel(const __grid_constant__ BfTable T, long long total, unsigned long long *counter) {
  extern __shared__ __align__(16) float2 smem[];
  __shared__ long long item_s;
  __shared__ int grp_s;
  // thread 0 takes the next item while the current one runs (the counter's latency stays hidden)
  long long nxt = threadIdx.x == 0 ? (long long)atomicAdd(counter, 1ull) : 0;
  for (;;) {
    if (threadIdx.x == 0) {
      const long long it = nxt;
      item_s = it;
      grp_s = it < total ? group_of(T, it) : 0;
      if (it < total) nxt = (long long)atomicAdd(counter, 1ull);
    }
    __syncthreads();
    const long long item = item_s;
    const int o = grp_s;
    __syncthreads();
    if (item >= total) break;
    const BfGroup &G = T.grp[o];
    const long long local = item - G.first_item;
    const int fc = (int)(local / G.per_fc), sub = (int)(local - (long long)fc * G.per_fc);
    if constexpr (V == 1) bf_few_item<OUT>(G.g, G.ct, G.out, fc, sub, smem);
    else if constexpr (V == 3) bf_many_item<OUT, 64>(G.g, G.ct, G.out, fc, sub, smem);
    else bf_many_item<OUT, 128>(G.g, G.ct, G.out, fc, sub, smem);
  }
}

template <int BT>
cudaError_t launch_many(const Geometry &g, int out_kind, const float2 *ct, void *out, cudaStream_t st) {
  const int nbt = (g.B + BT - 1) / BT;
  const long long ctas = (long long)g.F * kN * nbt;
  const size_t smem = (size_t)g.S * (BT + 2 * kP * kMC) * sizeof(float2);
  auto go = [&](auto kern) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)ctas, kManyThreads, smem, st>>>(g, ct, out, nbt);
    return cudaGetLastError();
  };
  switch (out_kind) {
    case OUT_VOLTAGES: return go(bf_many_kernel<OUT_VOLTAGES, BT>);
    case OUT_STOKES_I: return go(bf_many_kernel<OUT_STOKES_I, BT>);
    default: return go(bf_many_kernel<OUT_STOKES_IQUV, BT>);
  }
}

}  // namespace

cudaError_t launch_beamform(const Geometry &g, int variant, int out_kind, const float2 *ct, void *out,
                            cudaStream_t st) {
  if ((long long)g.F * kN == 0 || g.M == 0 || g.B == 0) return cudaSuccess;
  // Stokes I: 16 beams per CTA where that makes fewer passes per cost -- a 16-beam CTA costs ~1.91
  // of an 8-beam one (measured on the LOFAR block: the same reads, twice the arithmetic), so 9-16
  // and 25-32 beams gain 4-9 % and 17-24 would lose.  Voltages and IQUV keep 8 (their 16-beam
  // forms spill within two CTAs' registers per SM and lose to two 8-beam passes).
  if (variant == 1) {
    const bool wide = out_kind == OUT_STOKES_I && 191 * ((g.B + 15) / 16) < 100 * ((g.B + 7) / 8);
    return wide ? launch_few<16>(g, out_kind, ct, out, st) : launch_few<8>(g, out_kind, ct, out, st);
  }
  if (variant == 3) return launch_many<64>(g, out_kind, ct, out, st);
  return launch_many<128>(g, out_kind, ct, out, st);
}

namespace {

template <int V, int OUT>
cudaError_t launch_group_t(const BfTable &T, long long total, unsigned long long *counter, size_t smem,
                           cudaStream_t st) {
  auto kern = bf_group_kernel<V, OUT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // persistent: as many CTAs as are resident at once (registers and this launch's shared memory)
  int per_sm = 0, dev = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kManyThreads, smem);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  kern<<<per_sm * sms, kManyThreads, smem, st>>>(T, total, counter);
  return cudaGetLastError();
}

template <int V>
cudaError_t launch_group_v(int out_kind, const BfTable &T, long long total, unsigned long long *counter, size_t smem,
                           cudaStream_t st) {
  if (out_kind == OUT_STOKES_I) return launch_group_t<V, OUT_STOKES_I>(T, total, counter, smem, st);
  if (out_kind == OUT_STOKES_IQUV) return launch_group_t<V, OUT_STOKES_IQUV>(T, total, counter, smem, st);
  return launch_group_t<V, OUT_VOLTAGES>(T, total, counter, smem, st);
}

template <int V, int OUT>
int residency_t(size_t smem) {
  auto kern = bf_group_kernel<V, OUT>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kManyThreads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm;
}

template <int V>
int residency_v(int out_kind, size_t smem) {
  if (out_kind == OUT_STOKES_I) return residency_t<V, OUT_STOKES_I>(smem);
  if (out_kind == OUT_STOKES_IQUV) return residency_t<V, OUT_STOKES_IQUV>(smem);
  return residency_t<V, OUT_VOLTAGES>(smem);
}

}  // namespace

cudaError_t launch_bf_group(int variant, int out_kind, const BfGroup *h_groups, int ngrp, long long total,
                            unsigned long long *counter, size_t smem, cudaStream_t st) {
  if (total == 0) return cudaSuccess;
  if (ngrp < 1 || ngrp > kMaxGroups) return cudaErrorInvalidValue;
  BfTable T;
  T.n = ngrp;
  for (int i = 0; i < ngrp; ++i) T.grp[i] = h_groups[i];
  if (variant == 1) return launch_group_v<1>(out_kind, T, total, counter, smem, st);
  if (variant == 3) return launch_group_v<3>(out_kind, T, total, counter, smem, st);
  return launch_group_v<2>(out_kind, T, total, counter, smem, st);
}

int bf_group_residency(int variant, int out_kind, size_t smem) {
  if (variant == 1) return residency_v<1>(out_kind, smem);
  if (variant == 3) return residency_v<3>(out_kind, smem);
  return residency_v<2>(out_kind, smem);
}

int few_beams_per_item() { return kFewBeams; }
int many_beams_per_item(int variant) { return variant == 3 ? 64 : kBT; }
size_t bf_smem_bytes(int variant, int S) {
  if (variant == 1) return (size_t)S * kFewBeams * sizeof(float2);
  return (size_t)S * ((variant == 3 ? 64 : kBT) + 2 * kP * kMC) * sizeof(float2);
}

// Beam-former choice for AUTO: the few-beam kernel up to 32 beams (it reads the block once per 8
// beams at HBM speed; a 64-beam FP32 tile costs about as much as 6 such passes); beyond, the
// many-beam tile (128 or 64 beams per CTA) that leaves the fewest tile slots empty, a 64-beam slot
// counted as 1.15 of a 128-beam one (the narrower tile issues more shared loads per FMA).
int auto_bf_variant(int B, int S) {
  if (B <= 32 || S > many_beam_max_stations()) return 1;
  const double slots128 = (double)((B + 127) / 128) * 128.0;
  const double slots64 = (double)((B + 63) / 64) * 64.0 * 1.15;
  return slots64 < slots128 ? 3 : 2;
}

// Largest station count the many-beam kernel accepts (its shared memory holds S x (128 + 64) cf32).
int many_beam_max_stations() { return (227 * 1024) / ((kBT + 2 * kP * kMC) * (int)sizeof(float2)); }

}  // namespace lbf
