// 16-point DFT in registers, shared by the filter bank (256-point FFT as 16 x 16) and the
// 256-point channel-level dedispersion.
//
// Instruction choices: complex sums are packed FP32x2 adds; a difference x - y is one packed FMA
// y * (-1) + x, which is exact (the product is exact and the sum rounds once, as a subtraction
// does), so no separate negation is issued; products by -i and by the 45-degree twiddles are
// written out as adds and one packed multiply.
#pragma once

#include "lbf_internal.cuh"

namespace lbf {

// x - y as one packed FMA (exact: equal to the rounded difference).
__device__ __forceinline__ float2 sub2(float2 x, float2 y) {
  return __ffma2_rn(y, make_float2(-1.f, -1.f), x);
}

// In-place 4-point DFT, y_k = sum_n x_n exp(-2 pi i n k / 4).
__device__ __forceinline__ void dft4(float2 &x0, float2 &x1, float2 &x2, float2 &x3) {
  const float2 a = __fadd2_rn(x0, x2), b = sub2(x0, x2);
  const float2 c = __fadd2_rn(x1, x3), d = sub2(x1, x3);
  x0 = __fadd2_rn(a, c);
  x2 = sub2(a, c);
  x1 = make_float2(b.x + d.y, b.y - d.x);   // b - i d
  x3 = make_float2(b.x - d.y, b.y + d.x);   // b + i d
}

// The same with the third input multiplied by -i first: x2 -> (x2.y, -x2.x).
__device__ __forceinline__ void dft4_x2_times_minus_i(float2 &x0, float2 &x1, float2 &x2, float2 &x3) {
  const float2 a = make_float2(x0.x + x2.y, x0.y - x2.x);
  const float2 b = make_float2(x0.x - x2.y, x0.y + x2.x);
  const float2 c = __fadd2_rn(x1, x3), d = sub2(x1, x3);
  x0 = __fadd2_rn(a, c);
  x2 = sub2(a, c);
  x1 = make_float2(b.x + d.y, b.y - d.x);
  x3 = make_float2(b.x - d.y, b.y + d.x);
}

// a * exp(-2 pi i j / 16) for the j = n2 * k1 products of a 4 x 4 split other than 0 and 4.
__device__ __forceinline__ float2 tw16(float2 a, int j) {
  constexpr float c1 = 0.92387953251128674f, s1 = 0.38268343236508977f, r2 = 0.70710678118654752f;
  switch (j) {
    case 1: return cmul(a, make_float2(c1, -s1));
    case 2: return __fmul2_rn(make_float2(a.x + a.y, a.y - a.x), make_float2(r2, r2));     // r2 (1 - i)
    case 3: return cmul(a, make_float2(s1, -c1));
    case 6: return __fmul2_rn(make_float2(a.y - a.x, -a.x - a.y), make_float2(r2, r2));    // -r2 (1 + i)
    case 9: return cmul(a, make_float2(-c1, s1));
    default: return a;
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
    for (int k1 = 1; k1 < 4; ++k1)
      if (n2 * k1 != 4) a[4 * k1 + n2] = tw16(a[4 * k1 + n2], n2 * k1);
  dft4(a[0], a[1], a[2], a[3]);
  dft4(a[4], a[5], a[6], a[7]);
  dft4_x2_times_minus_i(a[8], a[9], a[10], a[11]);   // a[10] carries exp(-2 pi i 4 / 16) = -i
  dft4(a[12], a[13], a[14], a[15]);
  float2 t[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) t[r] = a[4 * (r & 3) + (r >> 2)];
#pragma unroll
  for (int r = 0; r < 16; ++r) a[r] = t[r];
}

}  // namespace lbf
