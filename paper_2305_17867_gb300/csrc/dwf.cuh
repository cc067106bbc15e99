// Double-word float ("float-float") arithmetic: a value is the unevaluated
// sum h + l of two floats with |l| <= ulp(h) / 2, about 48 significant bits.
// The mixed-precision modes run the M2M / L2L shifts of the upper tree in it
// instead of FP64: GB300 issues FP64 at 1/64 of the FP32 rate, and a
// double-word multiply-add takes about fifteen FP32 instructions.
//
// Building blocks (error-free transformations):
//  * TwoSum (Knuth, TAOCP vol. 2, 4.2.2; Moller 1965): s = fl(a + b) and the
//    exact rounding error e, a + b = s + e, in six additions;
//  * Fast2Sum (Dekker 1971): the same in three additions when |a| >= |b|;
//  * TwoProd by FMA: p = fl(a b), e = fma(a, b, -p), a b = p + e exactly.
// Sum of two double-words: TwoSum of the high parts, the low parts added to
// its error, renormalised by Fast2Sum (the "sloppy" double-word sum analysed
// by Joldes, Muller and Popescu, ACM TOMS 44(2), 2017).  Its error is at most
// about 4 u^2 (|x| + |y|) with u = 2^-24, i.e. 2^-46 (|x| + |y|): an absolute
// bound of the kind FP64 summation has (2^-53 (|x| + |y|)), with no relative
// bound when x and y cancel.  Product: TwoProd of the high parts plus the two
// cross terms by FMA, renormalised by Fast2Sum (the low x low term, below
// u^2 |x y|, is dropped): relative error at most about 4 u^2 = 2^-46.
// Every operation is written with the _rn intrinsics, which the compiler
// never contracts into an FMA or reorders: the transformations depend on each
// rounding taking place as written.
#pragma once

#include <cuda_runtime.h>

struct dwf {
  float h, l;
  __device__ __forceinline__ dwf() = default;
  __device__ __forceinline__ constexpr dwf(float hi, float lo) : h(hi), l(lo) {}
  __device__ __forceinline__ dwf(int v) : h((float)v), l(0.f) {}  // small integers (0, 1)
  __device__ __forceinline__ explicit dwf(double v) {
    h = __double2float_rn(v);
    l = __double2float_rn(__dsub_rn(v, (double)h));
  }
  __device__ __forceinline__ explicit operator double() const {
    return __dadd_rn((double)h, (double)l);
  }
};

__device__ __forceinline__ dwf dw_fast2sum(float a, float b) {  // |a| >= |b| (or a = 0)
  const float s = __fadd_rn(a, b);
  return dwf(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ dwf operator+(dwf x, dwf y) {
  const float s = __fadd_rn(x.h, y.h);
  const float bp = __fsub_rn(s, x.h);
  const float e = __fadd_rn(__fsub_rn(x.h, __fsub_rn(s, bp)), __fsub_rn(y.h, bp));
  return dw_fast2sum(s, __fadd_rn(e, __fadd_rn(x.l, y.l)));
}
__device__ __forceinline__ dwf operator-(dwf x) { return dwf(-x.h, -x.l); }
__device__ __forceinline__ dwf operator-(dwf x, dwf y) { return x + (-y); }
__device__ __forceinline__ dwf operator*(dwf x, dwf y) {
  const float p = __fmul_rn(x.h, y.h);
  float e = __fmaf_rn(x.h, y.h, -p);
  e = __fmaf_rn(x.h, y.l, e);
  e = __fmaf_rn(x.l, y.h, e);
  return dw_fast2sum(p, e);
}
__device__ __forceinline__ dwf& operator+=(dwf& x, dwf y) { return x = x + y; }
__device__ __forceinline__ dwf& operator-=(dwf& x, dwf y) { return x = x - y; }
__device__ __forceinline__ dwf& operator*=(dwf& x, dwf y) { return x = x * y; }
__device__ __forceinline__ dwf fma(dwf a, dwf b, dwf c) { return a * b + c; }
