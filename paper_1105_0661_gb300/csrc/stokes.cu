// Stand-alone Stokes I / IQUV with time integration (Sections 4.5 and 5.1), from beam voltages:
//   I = |X|^2 + |Y|^2, Q = |X|^2 - |Y|^2, U = 2 Re(X conj Y), V = 2 Im(X conj Y),
// each summed over Q consecutive spectra.  The general kernel has one CTA per (beam, subband,
// channel) row; lane l of a warp holds spectrum m, so the integration over Q <= 32 consecutive
// spectra is a warp-shuffle reduction and the voltage reads are fully coalesced.  Rows of a
// multiple of four spectra take a warp-per-row kernel with four spectra per lane (fewer shuffles
// and index operations per spectrum: the general kernel is instruction-bound).
#include "lbf_internal.cuh"

namespace lbf {
namespace {

__device__ __forceinline__ float stokes_value(int st, float2 X, float2 Y) {
  const float xx = fmaf(X.x, X.x, X.y * X.y);
  const float yy = fmaf(Y.x, Y.x, Y.y * Y.y);
  switch (st) {
    case 0: return xx + yy;
    case 1: return xx - yy;
    case 2: return 2.f * fmaf(X.x, Y.x, X.y * Y.y);
    default: return 2.f * fmaf(X.y, Y.x, -X.x * Y.y);
  }
}

template <int NS>
__global__ void __launch_bounds__(256)
stokes_kernel(Geometry g, const float2 *__restrict__ vol, float *__restrict__ out) {
  const long long row = blockIdx.x;                 // (b * F + f) * N + c
  const long long bf = row / kN;
  const int c = (int)(row - bf * kN);
  const int b = (int)(bf / g.F), f = (int)(bf - (long long)b * g.F);
  const float2 *vx = vol + (row * kP + 0) * g.M;
  const float2 *vy = vol + (row * kP + 1) * g.M;
  const int Mq = g.M / g.Q;
  // the loads of kPasses passes are issued before any of their arithmetic, so that each thread
  // keeps several requests in flight (the kernel is bound by DRAM latency x requests in flight)
  constexpr int kPasses = 4;
  for (int mb = 0; mb < g.M; mb += kPasses * blockDim.x) {
    float2 X[kPasses], Y[kPasses];
#pragma unroll
    for (int u = 0; u < kPasses; ++u) {
      const int m = mb + u * blockDim.x + threadIdx.x;
      X[u] = m < g.M ? vx[m] : make_float2(0.f, 0.f);
      Y[u] = m < g.M ? vy[m] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < kPasses; ++u) {
      const int m = mb + u * blockDim.x + threadIdx.x;
      if (mb + u * blockDim.x >= g.M) break;   // uniform across the CTA
      const bool active = m < g.M;
#pragma unroll
      for (int st = 0; st < NS; ++st) {
        float v = stokes_value(st, X[u], Y[u]);
        for (int o = 1; o < g.Q; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (active && (m & (g.Q - 1)) == 0)
          out[((((long long)b * NS + st) * g.F + f) * kN + c) * Mq + m / g.Q] = v;
      }
    }
  }
}

// Rows whose length M is a multiple of 4, in a 16-byte aligned buffer: one warp per row, lane l
// holding spectra 4u .. 4u + 3 of unit u = l + 32 k (two 16-byte loads per polarisation), so a lane
// sums four spectra itself and the integration over Q takes log2(Q / 4) shuffles per four spectra
// instead of log2(Q) per spectrum.
template <int NS>
__global__ void __launch_bounds__(256)
stokes4_kernel(Geometry g, const float2 *__restrict__ vol, float *__restrict__ out, long long rows) {
  const long long row = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (row >= rows) return;   // uniform across the warp
  const int lane = threadIdx.x & 31;
  const long long bf = row / kN;
  const int c = (int)(row - bf * kN);
  const int b = (int)(bf / g.F), f = (int)(bf - (long long)b * g.F);
  const float4 *vx = reinterpret_cast<const float4 *>(vol + (row * kP + 0) * g.M);
  const float4 *vy = reinterpret_cast<const float4 *>(vol + (row * kP + 1) * g.M);
  const int Mq = g.M / g.Q;
  const int units = g.M >> 2;
  const int qs = __ffs(g.Q) - 1;   // Q = 2^qs
  const int qu = g.Q >> 2;         // units per integration window (Q >= 4)
  float *orow[NS];
#pragma unroll
  for (int st = 0; st < NS; ++st) orow[st] = out + ((((long long)b * NS + st) * g.F + f) * kN + c) * Mq;
#pragma unroll 2
  for (int u0 = 0; u0 < units; u0 += 32) {
    const int u = u0 + lane;
    const bool active = u < units;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 x0 = active ? vx[2 * u] : z, x1 = active ? vx[2 * u + 1] : z;
    const float4 y0 = active ? vy[2 * u] : z, y1 = active ? vy[2 * u + 1] : z;
    const float2 X[4] = {make_float2(x0.x, x0.y), make_float2(x0.z, x0.w), make_float2(x1.x, x1.y), make_float2(x1.z, x1.w)};
    const float2 Y[4] = {make_float2(y0.x, y0.y), make_float2(y0.z, y0.w), make_float2(y1.x, y1.y), make_float2(y1.z, y1.w)};
#pragma unroll
    for (int st = 0; st < NS; ++st) {
      float v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = stokes_value(st, X[k], Y[k]);
      if (g.Q == 1) {
        if (active) {
#pragma unroll
          for (int k = 0; k < 4; ++k) orow[st][4 * u + k] = v[k];
        }
      } else if (g.Q == 2) {
        if (active) { orow[st][2 * u] = v[0] + v[1]; orow[st][2 * u + 1] = v[2] + v[3]; }
      } else {
        float sum = (v[0] + v[1]) + (v[2] + v[3]);
#pragma unroll
        for (int o = 1; o < 16; o <<= 1)
          if (o < qu) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (active && (u & (qu - 1)) == 0) orow[st][(4 * u) >> qs] = sum;
      }
    }
  }
}

}  // namespace

cudaError_t launch_stokes(const Geometry &g, int out_kind, const float2 *vol, float *out, cudaStream_t st) {
  const long long rows = (long long)g.B * g.F * kN;
  if (rows == 0 || g.M == 0) return cudaSuccess;
  if (g.M % 4 == 0 && (reinterpret_cast<uintptr_t>(vol) & 15) == 0) {
    const unsigned ctas = (unsigned)((rows + 7) / 8);
    if (out_kind == OUT_STOKES_IQUV)
      stokes4_kernel<4><<<ctas, 256, 0, st>>>(g, vol, out, rows);
    else
      stokes4_kernel<1><<<ctas, 256, 0, st>>>(g, vol, out, rows);
    return cudaGetLastError();
  }
  if (out_kind == OUT_STOKES_IQUV)
    stokes_kernel<4><<<(unsigned)rows, 256, 0, st>>>(g, vol, out);
  else
    stokes_kernel<1><<<(unsigned)rows, 256, 0, st>>>(g, vol, out);
  return cudaGetLastError();
}

}  // namespace lbf
