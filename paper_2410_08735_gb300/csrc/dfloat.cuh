// Double-float ("float-float") arithmetic for the refinement residual sweeps.
//
// A dfloat is the unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi) / 2: about 48
// significant bits, computed entirely on the FP32 pipe.  On this GPU the FP32 pipe runs many times the
// FP64 rate, so a sweep in dfloat arithmetic computes the residual b~ - A~ phi of the mixed-precision
// refinement to ~1e-14 relative accuracy at a fraction of the FP64 sweep's time.
//
// The operations rest on two error-free transformations (Dekker, "A floating-point technique for
// extending the available precision", Numer. Math. 18, 1971; Knuth, TAOCP vol. 2, 4.2.2):
//   two-sum:      s = fl(a + b), e = (a - (s - b')) + (b - b'), b' = s - a   gives a + b = s + e exactly;
//   two-product:  p = fl(a b), e = fma(a, b, -p)                              gives a b = p + e exactly.
// Addition adds the low parts to the error of the high-part two-sum and renormalises (the "sloppy" sum
// of Hida, Li and Bailey's double-double library, relative error a few units of 2^-48 of the larger
// operand); multiplication adds the cross terms hi*lo to the two-product's error.  Every rounding step
// uses a __f*_rn intrinsic: the compiler never contracts those into an FMA, which would break the
// transformations.
#pragma once
#include <cuda_runtime.h>

namespace rte {

struct dfloat {
  float hi, lo;
  dfloat() = default;
  __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr dfloat(int v) : hi((float)v), lo(0.f) {}
  __host__ __device__ constexpr dfloat(float v) : hi(v), lo(0.f) {}
  // nearest pair to a double: the FP64 arithmetic here runs once per constant, not per cell
  __host__ __device__ dfloat(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ dfloat df_renorm(float s, float e) {
  const float h = __fadd_rn(s, e);
  return dfloat(h, __fsub_rn(e, __fsub_rn(h, s)));
}

__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df_renorm(s, e);
}

__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }

__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_renorm(p, e);
}

__device__ __forceinline__ dfloat& operator+=(dfloat& a, dfloat b) { return a = a + b; }
__device__ __forceinline__ dfloat& operator*=(dfloat& a, dfloat b) { return a = a * b; }

}  // namespace rte
