// Float-float arithmetic (a value held as the unevaluated sum hi + lo of two
// FP32 numbers, about 48 significant bits) for the diagnostic reductions.
// GB300 issues FP64 at a small fraction of its FP32 rate, so the per-cell
// work of the FP64 global quantities runs in float-float and only per-column
// partial results are accumulated in FP64.  Error-free transformations:
// Knuth's TwoSum, Dekker's Fast2Sum (|a| >= |b|) and the FMA-based product
// error; the explicit _rn intrinsics keep the compiler from contracting or
// reassociating them.
#pragma once

namespace cfd {

struct FF {
  float hi, lo;
};

__device__ __forceinline__ FF ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ FF ff_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ FF ff_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ FF ff_add(FF x, FF y) {
  const FF s = ff_two_sum(x.hi, y.hi);
  return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

__device__ __forceinline__ FF ff_abs(FF x) { return x.hi < 0.f ? FF{-x.hi, -x.lo} : x; }

// x > y for normalised values (hi = fl(hi + lo))
__device__ __forceinline__ bool ff_gt(FF x, FF y) {
  return x.hi > y.hi || (x.hi == y.hi && x.lo > y.lo);
}

__device__ __forceinline__ double ff_to_double(FF x) { return (double)x.hi + (double)x.lo; }

// x^2 of a float-float value: hi^2 exact (TwoProd) plus 2 hi lo (lo^2 is
// below the result's precision).  Exact-product range: |hi| < kFFSquareMax.
constexpr float kFFSquareMax = 1e18f;
__device__ __forceinline__ FF ff_square(FF x) {
  if (!(fabsf(x.hi) < kFFSquareMax)) return FF{0.f, 0.f};  // the caller takes it in FP64
  FF s = ff_two_prod(x.hi, x.hi);
  s.lo = __fmaf_rn(2.f * x.hi, x.lo, s.lo);
  return ff_fast_two_sum(s.hi, s.lo);
}

// Per-cell contributions of a MAC velocity (x[c] at the cell's + faces,
// xm[c] at its - faces) to sum |u|^2 and to the divergence
// sum_c (x[c] - xm[c]) ih[c]: the squares and differences are exact, the
// products by ih keep their rounding error in lo.
__device__ __forceinline__ void ff_cell(const float (&x)[3], const float (&xm)[3],
                                        const float (&ih)[3], FF& sq, FF& div) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    sq = ff_add(sq, ff_two_prod(x[c], x[c]));
    const FF d = ff_two_sum(x[c], -xm[c]);
    FF t = ff_two_prod(d.hi, ih[c]);
    t.lo = __fmaf_rn(d.lo, ih[c], t.lo);
    div = c == 0 ? ff_fast_two_sum(t.hi, t.lo) : ff_add(div, t);
  }
}

}  // namespace cfd
