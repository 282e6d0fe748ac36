// FP64 helpers that keep work off the GB300's narrow FP64 pipe.
//
// Reciprocal and square root: a hardware seed (PTX rcp.approx.ftz.f64 /
// rsqrt.approx.ftz.f64, about 20 correct bits) refined by one third-order
// Newton-type step, i.e. the truncated binomial series
//   1/x        = y / (1 - e)     = y (1 + e + e^2 + ...),    e = 1 - x y
//   1/sqrt(x)  = y (1 - e)^(-1/2) = y (1 + e/2 + 3 e^2/8 + ...), e = 1 - x y^2
// which triples the number of correct bits (~60 > 53) in 3 FMAs (reciprocal)
// or 5 (square root, which reuses x*y). Results are within a few ulp of the
// correctly rounded values; the GPU tests check them against CUDA's 1/x and sqrt.
//
// Comparisons of non-negative doubles are done on their bit patterns as signed
// 64-bit integers, which orders them like the doubles and runs on the integer
// pipe. A negative or NaN operand compares as out of range, which the callers
// treat as an error.
#pragma once

#include <cstdint>

namespace pplbm {

__device__ __forceinline__ double rcp_seed(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  return y;
}

__device__ __forceinline__ double rsqrt_seed(double x) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  return y;
}

// 1/x for normal positive or negative x
__device__ __forceinline__ double fast_rcp(double x) {
  const double y = rcp_seed(x);
  const double e = fma(-x, y, 1.0);
  const double t = fma(e, e, e);
  return fma(y, t, y);
}

// sqrt(x) for normal positive x (NaN for x < 0)
__device__ __forceinline__ double fast_sqrt(double x) {
  const double y = rsqrt_seed(x);
  const double xy = x * y;
  const double e = fma(-xy, y, 1.0);
  const double t = fma(0.375, e, 0.5) * e;
  return fma(xy, t, xy);
}

__device__ __forceinline__ int64_t dbits(double x) { return __double_as_longlong(x); }

}  // namespace pplbm
