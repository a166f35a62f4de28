// Error-free transformations on binary32 (Knuth's TwoSum, TwoProduct by the FMA) and the
// compensated dot product built on them (Ogita, Rump and Oishi, "Accurate sum and dot product",
// SIAM J. Sci. Comput. 26 (2005), algorithm Dot2): a sum of products of binary32 numbers computed
// as if in twice the working precision and then rounded.  On this GPU binary32 runs on every lane
// at full rate while a binary64 instruction occupies its sub-partition's pipe for about 64 cycles,
// so long binary64 accumulations of binary32 products (the Gram matrix of the QR) are formed this
// way.  Every step uses round-to-nearest intrinsics, so the compiler cannot contract or
// reassociate the transformations.
#pragma once

#include <cuda_runtime.h>

namespace afq {

struct ff {   // hi + lo, unevaluated
  float hi, lo;
};

// s + e = a + b exactly (Knuth's TwoSum, six operations, no condition on the operands)
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return ff{s, e};
}
// p + e = a b exactly (barring underflow): the FMA returns the rounding error of the product
__device__ __forceinline__ ff ff_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return ff{p, __fmaf_rn(a, b, -p)};
}

// A running sum of products (Dot2): s the binary32 sum, c the gathered rounding errors of every
// product and every addition.  dot2_value() = s + c, rounded once to binary64.
struct dot2 {
  float s, c;
};
__device__ __forceinline__ void dot2_add(dot2& a, float x, float y) {   // a += x y
  const ff p = ff_two_prod(x, y);
  const ff t = ff_two_sum(a.s, p.hi);
  a.s = t.hi;
  a.c = __fadd_rn(a.c, __fadd_rn(p.lo, t.lo));
}
__device__ __forceinline__ double dot2_value(const dot2& a) { return (double)a.s + (double)a.c; }

}  // namespace afq
