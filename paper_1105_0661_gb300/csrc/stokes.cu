// Stand-alone Stokes I / IQUV with time integration (Sections 4.5 and 5.1), from beam voltages:
//   I = |X|^2 + |Y|^2, Q = |X|^2 - |Y|^2, U = 2 Re(X conj Y), V = 2 Im(X conj Y),
// each summed over Q consecutive spectra.  One CTA per (beam, subband, channel) row; lane l of a
// warp holds spectrum m, so the integration over Q <= 32 consecutive spectra is a warp-shuffle
// reduction and the voltage reads are fully coalesced.
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

}  // namespace

cudaError_t launch_stokes(const Geometry &g, int out_kind, const float2 *vol, float *out, cudaStream_t st) {
  const long long rows = (long long)g.B * g.F * kN;
  if (rows == 0 || g.M == 0) return cudaSuccess;
  if (out_kind == OUT_STOKES_IQUV)
    stokes_kernel<4><<<(unsigned)rows, 256, 0, st>>>(g, vol, out);
  else
    stokes_kernel<1><<<(unsigned)rows, 256, 0, st>>>(g, vol, out);
  return cudaGetLastError();
}

}  // namespace lbf
