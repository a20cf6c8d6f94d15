// Measured FP32 SIMT throughput of the current GPU: the denominator of the roofline of the FP32
// kernels that are bound by arithmetic (the many-beam beam former of Section 4.3, whose register
// kernel the paper itself quotes as a fraction of the FPU's peak).  A derived peak (SMs x lanes x
// clock) assumes a clock the kernel may not run at; this probe times dependent-free FMA chains on
// every SM with CUDA events, in the same process and at the same clocks as the kernel it rates.
#include "lbf.h"
#include "lbf_internal.cuh"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 16;        // independent FMA chains per thread: far more than the latency
constexpr int kProbeIters = 32768; // 2 x 16 x 32768 flop per thread per launch

// FFMA form: kChains scalar chains a = a * x + y.  x, y keep every chain bounded (x < 1).
__global__ void __launch_bounds__(kProbeThreads) ffma_probe_kernel(float *sink, int iters, float x, float y) {
  float a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = 1e-3f * (float)threadIdx.x + (float)i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], x, y);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == -1.0f) sink[blockIdx.x] = s;   // never true; keeps the chains live
}

// Packed FP32x2 form: kChains / 2 chains of (a0, a1) = (a0, a1) * (x, x) + (y, y).
__global__ void __launch_bounds__(kProbeThreads) ffma2_probe_kernel(float *sink, int iters, float x, float y) {
  float2 a[kChains / 2];
#pragma unroll
  for (int i = 0; i < kChains / 2; ++i) a[i] = make_float2(1e-3f * (float)threadIdx.x + i, (float)i + 0.5f);
  const float2 x2 = make_float2(x, x), y2 = make_float2(y, y);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains / 2; ++i) a[i] = __ffma2_rn(a[i], x2, y2);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains / 2; ++i) s += a[i].x + a[i].y;
  if (s == -1.0f) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" lbf_status lbf_measure_fp32_peak(int32_t reps, void *stream, lbf_alu_peak *out) {
  if (!out || reps < 1 || reps > 100) return LBF_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return LBF_ECUDA;
  cudaStream_t st = (cudaStream_t)stream;
  // four 256-thread CTAs per SM: 32 warps, 8 per scheduler, each with 16 independent chains
  const int ctas = 4 * sms;
  const double flop = 2.0 * kChains * (double)kProbeIters * kProbeThreads * ctas;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  double best[2] = {1e30, 1e30};
  for (int form = 0; form < 2 && e == cudaSuccess; ++form) {
    for (int r = 0; r <= reps && e == cudaSuccess; ++r) {   // r = 0 is a warm-up launch
      e = cudaEventRecord(a, st);
      if (form == 0) ffma_probe_kernel<<<ctas, kProbeThreads, 0, st>>>(nullptr, kProbeIters, 0.9999999f, 1e-7f);
      else ffma2_probe_kernel<<<ctas, kProbeThreads, 0, st>>>(nullptr, kProbeIters, 0.9999999f, 1e-7f);
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaEventRecord(b, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(b);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
      if (e == cudaSuccess && r > 0 && ms < best[form]) best[form] = ms;
    }
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (e != cudaSuccess) return LBF_ECUDA;
  out->sms = sms;
  out->ffma_ms = best[0];
  out->ffma2_ms = best[1];
  out->ffma_tflops = flop / (best[0] * 1e-3) / 1e12;
  out->ffma2_tflops = flop / (best[1] * 1e-3) / 1e12;
  return LBF_OK;
}
