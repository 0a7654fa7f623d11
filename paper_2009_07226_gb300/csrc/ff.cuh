// Unevaluated pairs of FP32 numbers (hi + lo) for the squared norms of the
// CG scalars.  GB300 runs FP64 arithmetic at a small fraction of its FP32
// rate, so sums of squares are formed and reduced in pairs of FP32 values and
// converted to FP64 once per partial sum.  The square of an FP32 value is
// exact as a pair (the error of the rounded product, by one FMA), and pairs
// are added with Knuth's TwoSum on the high parts: about 2^-48 relative error
// per addition, close to an FP64 accumulator (2^-53) and far below the FP32
// rounding of the vectors themselves.
#pragma once

namespace xct {

struct FF {
  float hi, lo;
};

// v * v exactly: hi = RN(v*v), lo = v*v - hi (FMA)
__device__ __forceinline__ FF ff_sq(float v) {
  const float h = v * v;
  return FF{h, fmaf(v, v, -h)};
}

// a + b: TwoSum of the high parts, low parts and the rounding error added,
// renormalised
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bv = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bv)), __fsub_rn(b.hi, bv));
  const float lo = __fadd_rn(__fadd_rn(a.lo, b.lo), err);
  const float h = __fadd_rn(s, lo);
  return FF{h, __fsub_rn(lo, __fsub_rn(h, s))};
}

__device__ __forceinline__ FF ff_shfl_xor(FF a, int o) {
  return FF{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}

__device__ __forceinline__ double ff_to_double(FF a) { return (double)a.hi + (double)a.lo; }

}  // namespace xct
