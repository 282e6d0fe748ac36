// Sums of a few doubles on the integer pipe in one fixed-point frame.
//
// The step's sums (the density moments of Eqs. Density and Momentum over the nine
// populations; the Shan-Chen stencil of Eq. ShanChenForce over the eight neighbours'
// psi) add values of one sign class and similar size. Each sum here aligns all its
// operands once to the largest exponent among them, adds them as 64-bit integers
// (exact and associative) and rounds the integer sum once to a double:
//
//   operand x = s 2^(e - 1075), s the 53-bit significand, e the biased exponent;
//   left-aligned significand L = s 2^11 (leading one at bit 63), x = L 2^(e - 1086);
//   in a frame with top exponent eg = max e + G, the term of x is
//     t = floor(L / 2^(eg - e)),  x ~ t 2^(eg - 1086),
//   so the G high bits of every term are zero (room for the sum to grow) and the
//   largest operand keeps all its bits with 11 - G bits below them; a smaller operand
//   loses only the bits below the frame's bit 0.
//
// The integer sum S of the terms is then rounded to nearest (ties to even) as a
// double with exponent eg - clz(S). The result is within half an ulp plus
// (number of operands) x 2^(G - 11) ulp of the largest operand of the exact sum
// (the truncated bits), i.e. within 0.57 ulp for a sum of nine positive operands.
// Against a chain of IEEE additions (a rounding per addition) it costs a fraction
// of the integer instructions of the software additions of fp64.cuh and keeps the
// FP64 pipe, the step's bottleneck, free; symmetric operand sets give exactly
// cancelling sums (integer addition is associative).
//
// Domain: positive normal finite operands below 2^1008 (callers test them, or
// rely on the density pass's error word, which flags any non-finite or non-positive
// psi^2). Results below 2^-1022 flush to a zero of their sign.
//
// The functions compile for the host as well, so that a CPU test can compare them
// with exact rational sums.
#pragma once

#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define PPLBM_FX __host__ __device__ __forceinline__
#else
#define PPLBM_FX inline
#endif

namespace pplbm {
namespace fx {

typedef unsigned long long u64;
typedef long long i64;

// headroom bits of a frame: sums of up to 16 terms (or 12 after the stencil's
// factor 4 on four of them) cannot overflow 64 bits
constexpr int kG = 4;

// bit pattern of a double and back, through an opaque move on the device so that
// the optimiser keeps the integer work on the integer pipe
PPLBM_FX u64 bits_of(double x) {
#ifdef __CUDA_ARCH__
  u64 r;
  asm("mov.b64 %0, %1;" : "=l"(r) : "d"(x));
  return r;
#else
  u64 r;
  std::memcpy(&r, &x, sizeof(r));
  return r;
#endif
}

PPLBM_FX double double_of(u64 r) {
#ifdef __CUDA_ARCH__
  double x;
  asm("mov.b64 %0, %1;" : "=d"(x) : "l"(r));
  return x;
#else
  double x;
  std::memcpy(&x, &r, sizeof(x));
  return x;
#endif
}

PPLBM_FX unsigned hi32(u64 b) { return (unsigned)(b >> 32); }

PPLBM_FX int clz64(u64 v) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)v);
#else
  return v ? __builtin_clzll(v) : 64;
#endif
}

// top exponent of a frame from the largest high word of its (positive) operands
PPLBM_FX int frame_top(unsigned max_hi) { return (int)(max_hi >> 20) + kG; }

// The term of the positive normal double with bit pattern b in the frame with top
// exponent eg, multiplied by 2^UP (UP <= kG, an exact factor 2^UP on the operand).
template <int UP = 0>
PPLBM_FX u64 term(u64 b, int eg) {
  const int d = eg - UP - (int)(b >> 52);  // >= kG - UP >= 0
  const u64 l = (b << 11) | (1ull << 63);
  return l >> (d < 63 ? d : 63);
}

// The double nearest (ties to even) to s 2^(eg - 1086), s >= 0; +0 for s = 0 or a
// result below 2^-1022.
PPLBM_FX u64 round_frame_u(u64 s, int eg) {
  const int lz = clz64(s);      // 0..64
  const u64 n = s << (lz & 63);  // leading one at bit 63 (0 for s = 0)
  u64 m = n >> 11;               // 53-bit significand
  const unsigned low = (unsigned)n & 0x7FFu;
  m += (u64)((low > 0x400u) | ((low == 0x400u) & (unsigned)(m & 1)));
  const int er = eg - lz;  // biased exponent (a carry of the rounding moves into it)
  const u64 r = ((u64)(i64)er << 52) + (m - (1ull << 52));
  return (s == 0 || er <= 0) ? 0ull : r;
}

// The same for a signed integer sum s (two's complement): +0 for s = 0.
PPLBM_FX u64 round_frame_s(i64 s, int eg) {
  const u64 sg = (u64)s & (1ull << 63);
  const u64 a = sg ? (u64)0 - (u64)s : (u64)s;
  return round_frame_u(a, eg) | sg;
}

// The Shan-Chen stencil sums 12 sum_i w(|c_i|^2) psi(x + c_i) c_i of Eq.
// ShanChenForce (w = 1/3 on the axes, 1/12 on the diagonals), i.e.
//   gx = 4 (pE - pW) + (pNE - pSW) + (pSE - pNW),
//   gy = 4 (pN - pS) + (pNE - pSW) - (pSE - pNW),
// from the eight neighbours' psi (positive finite values below 2^1008; a zero or
// subnormal operand counts as at most one unit of the frame's bit 0), each exact in
// one frame and rounded once. An infinite, NaN or negative operand gives NaN.
PPLBM_FX void shan_chen_stencil(double pE, double pW, double pN, double pS, double pNE, double pNW, double pSW,
                                double pSE, double* gx, double* gy) {
  const u64 bE = bits_of(pE), bW = bits_of(pW), bN = bits_of(pN), bS = bits_of(pS);
  const u64 bNE = bits_of(pNE), bNW = bits_of(pNW), bSW = bits_of(pSW), bSE = bits_of(pSE);
  unsigned mx = hi32(bE);
  mx = mx > hi32(bW) ? mx : hi32(bW);
  mx = mx > hi32(bN) ? mx : hi32(bN);
  mx = mx > hi32(bS) ? mx : hi32(bS);
  mx = mx > hi32(bNE) ? mx : hi32(bNE);
  mx = mx > hi32(bNW) ? mx : hi32(bNW);
  mx = mx > hi32(bSW) ? mx : hi32(bSW);
  mx = mx > hi32(bSE) ? mx : hi32(bSE);
  const int eg = frame_top(mx);
  const bool bad = mx >= 0x7FF00000u;
  // |4 (pE - pW)| < 2^(66 - kG) and each diagonal difference < 2^(64 - kG): the sums
  // stay below 2^63
  const u64 d1 = term(bNE, eg) - term(bSW, eg);
  const u64 d2 = term(bSE, eg) - term(bNW, eg);
  const u64 ex = term<2>(bE, eg) - term<2>(bW, eg);
  const u64 ny = term<2>(bN, eg) - term<2>(bS, eg);
  const u64 nan = 0x7FF8000000000000ull;
  *gx = double_of(bad ? nan : round_frame_s((i64)(ex + d1 + d2), eg));
  *gy = double_of(bad ? nan : round_frame_s((i64)(ny + d1 - d2), eg));
}

// Density moments of nine populations f0..f8 (D2Q9 order: rest, E, N, W, S, NE, NW,
// SW, SE), all positive normal below 2^1008 (callers test that with
// positive_normal_range): rho = sum f (Eq. Density), j = sum f c (Eq. Momentum)
// and, when STRESS, the second moments of rows 7 and 8 of Eq. MatrixMRT,
// (f1 + f3) - (f2 + f4) and (f5 + f7) - (f6 + f8); eg = frame_top(max high word).
template <bool STRESS>
PPLBM_FX void density_moments(const double (&f)[9], int eg, double* rho, double* jx, double* jy, double* m7,
                              double* m8) {
  u64 t[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) t[k] = term(bits_of(f[k]), eg);
  // each term < 2^(64 - kG): the nine-term sum stays below 2^64, the signed ones
  // below 2^63 in magnitude
  const u64 sxp = t[1] + t[5] + t[8], sxm = t[3] + t[6] + t[7];  // c_x = +1, -1
  const u64 syp = t[2] + t[5] + t[6], sym = t[4] + t[7] + t[8];  // c_y = +1, -1
  *rho = double_of(round_frame_u(t[0] + t[2] + t[4] + sxp + sxm, eg));
  *jx = double_of(round_frame_s((i64)(sxp - sxm), eg));
  *jy = double_of(round_frame_s((i64)(syp - sym), eg));
  if (STRESS) {
    *m7 = double_of(round_frame_s((i64)((t[1] + t[3]) - (t[2] + t[4])), eg));
    *m8 = double_of(round_frame_s((i64)((t[5] + t[7]) - (t[6] + t[8])), eg));
  }
}

// True if all K values are positive normal doubles below 2^1008 (high words in
// [0x00100000, 0x7EF00000): a negative value's high word is above the range); the
// largest high word goes to *max_hi.
template <int K>
PPLBM_FX bool positive_normal_range(const double (&v)[K], unsigned* max_hi) {
  unsigned mn = 0xFFFFFFFFu, mx = 0u;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const unsigned h = hi32(bits_of(v[k]));
    mn = mn < h ? mn : h;
    mx = mx > h ? mx : h;
  }
  *max_hi = mx;
  return mn >= 0x00100000u && mx < 0x7EF00000u;
}

}  // namespace fx
}  // namespace pplbm
