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
// treat as an error. add_pos_int and add_int are software IEEE additions on the
// integer pipe, bit for bit equal to the FP64 pipe's: add_int carries the sums the
// fixed-point frames of fixsum.cuh do not (the surface-tension path, the adjoint's
// remaining sums, the FD solver's one-sided differences); the issue-rate probe times
// add_pos_int.
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

// Bit patterns in and out through an opaque move, so that the optimiser does not
// recognise the integer masks below as FP64 operations (an AND with ~sign is fabs, an
// XOR of the sign is a negation) and move them back onto the FP64 pipe.
__device__ __forceinline__ unsigned long long opaque_bits(double x) {
  unsigned long long r;
  asm("mov.b64 %0, %1;" : "=l"(r) : "d"(x));
  return r;
}
__device__ __forceinline__ double opaque_double(unsigned long long r) {
  double x;
  asm("mov.b64 %0, %1;" : "=d"(x) : "l"(r));
  return x;
}

// Sum of two positive normal doubles on the integer pipe, correctly rounded
// (round to nearest, ties to even: IEEE 754-2008, 4.3.1), so bitwise equal to the
// FP64 pipe's x + y. The integer pipe runs beside the narrow FP64 pipe, so an
// addition moved here frees an FP64 issue slot.
// Textbook method (e.g. Muller et al., Handbook of Floating-Point Arithmetic, ch. 7):
// align the smaller significand with three extra bits (guard, round and a sticky bit
// that ORs everything shifted out), add, renormalise by at most one place, round.
// Both operands must be positive and normal with a normal sum;
// pplbm_int_add_selftest compares it with the FP64 add bit for bit.
__device__ __forceinline__ double add_pos_int(double x, double y) {
  typedef unsigned long long u64;
  const u64 a = opaque_bits(x), b = opaque_bits(y);
  const u64 hi = a > b ? a : b, lo = a > b ? b : a;  // positive doubles order like their bits
  const int eh = (int)(hi >> 52);
  const int d = min(eh - (int)(lo >> 52), 63);
  const u64 H = 1ull << 52, M = H - 1;
  const u64 mh = ((hi & M) | H) << 3;  // significands with 3 extra bits, < 2^56
  const u64 ml = ((lo & M) | H) << 3;
  const u64 sh = ml >> d;
  u64 m = mh + (sh | (u64)((sh << d) != ml));  // the sticky bit: anything shifted out
  const u64 ov = m >> 56;                         // 1 if the sum carried into bit 56
  m = (m >> ov) | (m & ov);
  const u64 low = m & 7;                          // guard, round, sticky
  m >>= 3;
  m += (low > 4) | ((low == 4) & (m & 1));        // ties to even
  // a carry out of the significand (m == 2^53) moves into the exponent field
  return opaque_double((((u64)(eh + (int)ov)) << 52) + (m - H));
}

// The sum of the doubles with bit patterns a and b on the integer pipe, correctly
// rounded (round to nearest, ties to even), for normal or zero operands whose sum is
// normal or zero: then bitwise the FP64 pipe's sum (including +0 for an exact
// cancellation and the signs of zero sums). Same method as add_pos_int, with the
// magnitudes subtracted when the signs differ: the three extra bits then also cover
// the one-place left shift a subtraction of operands two or more binades apart can
// need; operands closer than that lose no bit when aligned, so a cancellation is exact
// and renormalised by the leading-zero count. Outside that domain it does not call
// the FP64 pipe (a fallback there would be computed speculatively and cost the FP64
// issue slots this exists to save): a subnormal operand counts as zero, a result below
// 2^-1022 flushes to a signed zero, and an infinite or NaN operand gives a NaN. The
// step's quantities stay far from that range (densities, psi and velocities are above
// 1e-300 or exactly zero).
__device__ __forceinline__ double add_bits_int(unsigned long long a, unsigned long long b) {
  typedef unsigned long long u64;
  const u64 S = 1ull << 63, H = 1ull << 52, M = H - 1;
  const u64 ua = a & ~S, ub = b & ~S;
  const bool sw = ub > ua;
  const u64 big = sw ? b : a;
  const u64 uh = sw ? ub : ua, ul = sw ? ua : ub;
  const u64 sign = big & S;
  const int eh = (int)(uh >> 52), el = (int)(ul >> 52);
  const int d = min(eh - el, 63);
  const u64 mh = ((uh & M) | H) << 3, ml = ((ul & M) | H) << 3;
  const u64 sh = ml >> d;
  const u64 al = sh | (u64)((sh << d) != ml);
  u64 m = ((a ^ b) & S) ? mh - al : mh + al;  // < 2^57
  // bring the leading one to bit 55: one place right after a carry, or left by the
  // leading zeros after a cancellation
  const int lz = __clzll((long long)m) - 8;  // -1 (carry) .. 56 (m = 0)
  const u64 mr = (m >> 1) | (m & 1), mlft = m << (lz < 0 ? 0 : lz);
  m = lz < 0 ? mr : mlft;
  const int e = lz < 0 ? eh + 1 : eh - lz;
  const u64 low = m & 7;
  m >>= 3;
  m += (low > 4) | ((low == 4) & (m & 1));
  u64 r = sign | ((((u64)e) << 52) + (m - H));
  r = e <= 0 ? sign : r;                        // underflow: signed zero
  r = lz == 56 ? 0ull : r;                      // exact cancellation: +0
  r = el == 0 ? (uh == 0 ? (a & b) : big) : r;  // smaller operand zero (or subnormal)
  r = eh == 2047 ? 0x7FF8000000000000ull : r;   // infinite or NaN operand
  return opaque_double(r);
}

// x + y and x - y on the integer pipe (add_bits_int; the sign of y flipped in its bits)
__device__ __forceinline__ double add_int(double x, double y) { return add_bits_int(opaque_bits(x), opaque_bits(y)); }
__device__ __forceinline__ double sub_int(double x, double y) {
  return add_bits_int(opaque_bits(x), opaque_bits(y) ^ (1ull << 63));
}

}  // namespace pplbm
