// 16-point DFT in registers, shared by the filter bank (256-point FFT as 16 x 16) and the
// 256-point channel-level dedispersion.  Packed FP32x2 adds for the butterflies.
#pragma once

#include "lbf_internal.cuh"

namespace lbf {

__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }

// In-place 4-point DFT, y_k = sum_n x_n exp(-2 pi i n k / 4), packed FP32x2 adds.
__device__ __forceinline__ void dft4(float2 &x0, float2 &x1, float2 &x2, float2 &x3) {
  const float2 a = __fadd2_rn(x0, x2), b = __fadd2_rn(x0, f2neg(x2));
  const float2 c = __fadd2_rn(x1, x3), d = __fadd2_rn(x1, f2neg(x3));
  x0 = __fadd2_rn(a, c);
  x2 = __fadd2_rn(a, f2neg(c));
  x1 = __fadd2_rn(b, make_float2(d.y, -d.x));   // b - i d
  x3 = __fadd2_rn(b, make_float2(-d.y, d.x));   // b + i d
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

}  // namespace lbf
