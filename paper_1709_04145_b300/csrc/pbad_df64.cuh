// Double-float ("df64") arithmetic: a value is the unevaluated sum hi + lo
// of two binary32 numbers (|lo| <= ulp(hi)/2), about 48 significant bits,
// computed on the binary32 pipes. Built from the error-free transformations
// of Knuth (two-sum), Dekker (fast two-sum) and the FMA two-product, as in
// Dekker's 1971 double-length arithmetic. Used by the optional double-float
// residual pass of the link-parallel mapping (pbad_lp.cuh).
//
// The compiler may not reassociate binary32 additions (no fast-math
// flags), and every product whose rounding error matters goes through an
// explicit fmaf.
#pragma once
#include <cuda_runtime.h>

namespace pbad {

struct df64 {
  float hi, lo;
};

__device__ __forceinline__ df64 df_from(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double df_to(df64 a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ df64 df_zero() { return {0.0f, 0.0f}; }

// a + b = s + e exactly (Knuth)
__device__ __forceinline__ df64 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
// the same when |a| >= |b| (Dekker)
__device__ __forceinline__ df64 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df64 df_add(df64 a, df64 b) {
  df64 s = two_sum(a.hi, b.hi);
  const df64 t = two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df64 df_neg(df64 a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df64 df_sub(df64 a, df64 b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df64 df_mul(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);  // exact error of the product
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ df64 df_fma(df64 a, df64 b, df64 c) { return df_add(df_mul(a, b), c); }
__device__ __forceinline__ df64 df_shfl(df64 v, int src) {
  return {__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
}

// C = A B for affine 3x4 matrices (implicit bottom row 0 0 0 1)
__device__ __forceinline__ void df_compose(const df64* A, const df64* B, df64* C) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
      C[4 * r + c] = df_fma(A[4 * r], B[c], df_fma(A[4 * r + 1], B[4 + c], df_mul(A[4 * r + 2], B[8 + c])));
    C[4 * r + 3] = df_fma(A[4 * r], B[3], df_fma(A[4 * r + 1], B[7], df_fma(A[4 * r + 2], B[11], A[4 * r + 3])));
  }
}
__device__ __forceinline__ void df_cross(const df64* a, const df64* b, df64* c) {
  c[0] = df_sub(df_mul(a[1], b[2]), df_mul(a[2], b[1]));
  c[1] = df_sub(df_mul(a[2], b[0]), df_mul(a[0], b[2]));
  c[2] = df_sub(df_mul(a[0], b[1]), df_mul(a[1], b[0]));
}

}  // namespace pbad
