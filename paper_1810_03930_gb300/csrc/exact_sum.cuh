// Sums of exact FP32 products without FP64 multiplies (GB300 executes FP64 at 1/64 of the FP32
// rate), for the FP64 Gram and Q = X R^{-1} of the final orthonormalisation.
//
// Each product x y is split exactly, x y = h + r with h = fl(x y), r = fma(x, y, -h)
// (TwoProduct), and summed as in Ogita, Rump and Oishi's Dot2 in three levels:
//   a segment of kExactSeg terms:  s += h by TwoSum (exact), its errors into e, the product
//                                   errors r into their own sum (added to e first, r is lost
//                                   against the larger e, and the r of squares are not centred:
//                                   a diagonal of X^T X then drifts by a few u^2, u = 2^-24);
//   kExactSeg2 segments:           S += s by TwoSum, its errors and e into E, r into R;
//   then into a double total.
// On CPU emulation with 64 and 16 the relative error of a sum of squares is -1.7e-16 +- 5e-16,
// as good as flushing every segment into double, with a sixteenth of the FP64 additions.
#pragma once

namespace plam {

constexpr int kExactSeg = 64;    // terms per first-level segment
constexpr int kExactSeg2 = 16;   // segments per second-level block

struct ExactAcc {
  float s, e, r;      // the running segment
  float S, E, R;      // the running block of segments
  double tot;         // the blocks
};

__device__ __forceinline__ void exact_zero(ExactAcc& a) {
  a.s = a.e = a.r = 0.f;
  a.S = a.E = a.R = 0.f;
  a.tot = 0.0;
}

// TwoSum: s + err = a + b exactly.
__device__ __forceinline__ float two_sum(float a, float b, float& err) {
  const float s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
  return s;
}

// One term h + r (h the rounded product, r its exact error, or any small companion term).
__device__ __forceinline__ void exact_add(ExactAcc& a, float h, float r) {
  float q;
  a.s = two_sum(a.s, h, q);
  a.e = __fadd_rn(a.e, q);
  a.r = __fadd_rn(a.r, r);
}

// End of a segment.
__device__ __forceinline__ void exact_seg(ExactAcc& a) {
  float q;
  a.S = two_sum(a.S, a.s, q);
  a.E = __fadd_rn(a.E, __fadd_rn(q, a.e));
  a.R = __fadd_rn(a.R, a.r);
  a.s = a.e = a.r = 0.f;
}

// End of a block of segments.
__device__ __forceinline__ void exact_block(ExactAcc& a) {
  a.tot += (double)a.S + ((double)a.E + (double)a.R);
  a.S = a.E = a.R = 0.f;
}

__device__ __forceinline__ double exact_value(const ExactAcc& a) {
  return a.tot + ((double)a.S + ((double)a.E + (double)a.R)) +
         ((double)a.s + ((double)a.e + (double)a.r));
}

}  // namespace plam
