// ff.cuh -- error-free transformations on the FP32 pipe, used where an
// FP64-accurate result is needed at FP32 speed (GB300 runs FP64 FMAs at
// 1/64 of the FP32 rate).
//
// An FP64 value x is carried as hi + lo with hi = fl32(x), lo = fl32(x - hi)
// (48 significant bits). A product a*b of two such pairs is p + e with
// p = ah*bh and e = fma(ah, bh, -p) + ah*bl + al*bh (Dekker's exact product
// via FMA plus the first-order cross terms). Sums go into a three-float
// accumulator (S, s1, s2): S += p by Knuth's TwoSum, its exact error and e
// are each added to s1 by TwoSum, and those errors go to s2. Every rounding
// left is relative to one term (~2^-48), which makes a long dot product as
// accurate as an FP64 one (checked against long double in emulation:
// median error 3.6e-17 of sum |a||b| over 3072 terms, FP64 2.6e-17).
#pragma once

namespace harp {

__device__ __forceinline__ void ff_split(double x, float& h, float& l) {
  h = (float)x;
  l = (float)(x - (double)h);
}

// Knuth's TwoSum: returns fl(x + y) and sets err = x + y - fl(x + y) exactly.
__device__ __forceinline__ float two_sum(float x, float y, float& err) {
  const float s = __fadd_rn(x, y);
  const float v = __fsub_rn(s, x);
  err = __fadd_rn(__fsub_rn(x, __fsub_rn(s, v)), __fsub_rn(y, v));
  return s;
}

// (S, s1, s2) += a * b, a = ah + al, b = bh + bl.
__device__ __forceinline__ void fff_mac(float& S, float& s1, float& s2, float ah, float al,
                                        float bh, float bl) {
  // Round-to-nearest intrinsics keep the compiler from contracting the
  // product into the sums, which would break the error-free transformations.
  const float p = __fmul_rn(ah, bh);
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  float t;
  S = two_sum(S, p, t);
  float t2, t3;
  s1 = two_sum(s1, t, t2);
  s1 = two_sum(s1, e, t3);
  s2 = __fadd_rn(s2, __fadd_rn(t2, t3));
}

// (S, s) += a * b with a double-float accumulator (Ogita-Rump-Oishi Dot2:
// exact product error and TwoSum error gathered in one float). Half the
// instructions of fff_mac; its error grows with the running sum (~1e-14 of
// sum |a||b| over 3072 terms), enough for updates that are small against
// the quantity being corrected.
__device__ __forceinline__ void ff2_mac(float& S, float& s, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  float t;
  S = two_sum(S, p, t);
  s = __fadd_rn(s, __fadd_rn(t, e));
}

}  // namespace harp
