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

// Frames take operands below 2^1008 (high word below 0x7EF00000, magnitudes): with
// at most 8 bits of headroom no rounded result can then overflow the exponent. An
// operand at or above it, or infinite or NaN, makes the frame's results NaN.
constexpr unsigned kFrameMaxHi = 0x7EF00000u;
constexpr unsigned long long kNaN = 0x7FF8000000000000ull;

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
// one frame and rounded once. A negative operand, or one out of the frames' range,
// gives NaN.
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
  const bool bad = mx >= kFrameMaxHi;
  // |4 (pE - pW)| < 2^(66 - kG) and each diagonal difference < 2^(64 - kG): the sums
  // stay below 2^63
  const u64 d1 = term(bNE, eg) - term(bSW, eg);
  const u64 d2 = term(bSE, eg) - term(bNW, eg);
  const u64 ex = term<2>(bE, eg) - term<2>(bW, eg);
  const u64 ny = term<2>(bN, eg) - term<2>(bS, eg);
  const u64 nan = kNaN;
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

// The term of a double of either sign (bit pattern b) in the frame with top exponent
// eg, rounded to the nearest unit (halves away from zero) rather than truncated, so
// that the terms' errors do not all lean one way; zero gives 0. Needs eg - e >= 1 for
// the operand's biased exponent e (frames built with a headroom of at least 1).
PPLBM_FX i64 sterm(u64 b, int eg) {
  const int e = (int)((b >> 52) & 0x7FFu);
  const int d = eg - e - 1;  // >= 0: one place more than the term, then round
  const u64 l = (b << 11) | ((u64)(e != 0) << 63);
  const u64 m = ((l >> (d < 63 ? d : 63)) + 1) >> 1;
  const u64 neg = (u64)((i64)b >> 63);  // 0 or all ones
  return (i64)((m ^ neg) - neg);
}

// high word of a double with its sign cleared: the magnitude's order
PPLBM_FX unsigned mag_hi(u64 b) { return hi32(b) & 0x7FFFFFFFu; }

// j + h, j + 2 h, j + 3 h and, when MINUS, j - h: exact in one frame, each rounded
// once (for J = j + F/2 = rho u of Eq. Momentum, P = j + F, P + F/2 and j - F/2, with
// h = F/2). Operands out of the frames' range give NaN.
template <bool MINUS>
PPLBM_FX void j_h_combos(double j, double h, double* jh, double* j2h, double* j3h, double* jmh) {
  const u64 bj = bits_of(j), bh = bits_of(h);
  const unsigned mj = mag_hi(bj), mh = mag_hi(bh);
  const unsigned mx = mj > mh ? mj : mh;
  const int eg = frame_top(mx);  // |j| + 3 |h| < 4 2^(64 - kG) = 2^62
  const u64 tj = (u64)sterm(bj, eg), th = (u64)sterm(bh, eg);
  const u64 s1 = tj + th, s2 = s1 + th;
  const bool bad = mx >= kFrameMaxHi;
  *jh = double_of(bad ? kNaN : round_frame_s((i64)s1, eg));
  *j2h = double_of(bad ? kNaN : round_frame_s((i64)s2, eg));
  *j3h = double_of(bad ? kNaN : round_frame_s((i64)(s2 + th), eg));
  if (MINUS) *jmh = double_of(bad ? kNaN : round_frame_s((i64)(tj - th), eg));
}

// headroom of the collision output frame: the largest combination below has
// coefficients summing to 44 < 2^6, plus the sign
constexpr int kGOut = 7;

// Post-collision populations f*_0..8 of the reduced collision (Lambda = I, or with
// rows 7, 8 relaxing at omega = 1/tau(rho) when SHEAR): with every input scaled by
// 1/36 except zz,
//   r = rho/36, xx = Pi_xx/36, yy = Pi_yy/36, xy = Pi_xy/36 (the unit-tau second
//   moments u (P + F/2) and u_x P_y + u_y F_x/2), px = P_x/36, py = P_y/36 (P = j + F),
//   zz = the Li term sigma |F|^2 / (3 psi^2), and for SHEAR p7 = (1 - omega) A7/36,
//   p8 = (1 - omega) A8/36 (the rows 7, 8 corrections),
// the populations w_i [rho + 3 c_i.P + 4.5 (c_i c_i - I/3) : Pi*] + zz (-8, 1, ..., 1)
// are small-integer combinations:
//   f1,3 = 4 r + 12 xx - 6 yy + 9 p7 + zz +- 12 px,  f2,4 = 4 r - 6 xx + 12 yy - 9 p7 + zz +- 12 py,
//   f5,7 = B + 9 (xy + p8) +- 3 (px + py),            f6,8 = B - 9 (xy + p8) +- 3 (py - px),
//   B = r + 3 (xx + yy) + zz,                         f0 = 4 (4 r - 6 (xx + yy) - 2 zz),
// evaluated exactly in one frame over the seven (nine) inputs and each rounded once.
// An input out of the frames' range makes every population NaN.
template <bool SHEAR>
PPLBM_FX void reduced_populations(double r, double xx, double yy, double xy, double px, double py, double zz,
                                  double p7, double p8, double (&f)[9]) {
  const u64 br = bits_of(r), bxx = bits_of(xx), byy = bits_of(yy), bxy = bits_of(xy);
  const u64 bpx = bits_of(px), bpy = bits_of(py), bz = bits_of(zz);
  const u64 b7 = SHEAR ? bits_of(p7) : 0ull, b8 = SHEAR ? bits_of(p8) : 0ull;
  unsigned mx = mag_hi(br);
  mx = mx > mag_hi(bxx) ? mx : mag_hi(bxx);
  mx = mx > mag_hi(byy) ? mx : mag_hi(byy);
  mx = mx > mag_hi(bxy) ? mx : mag_hi(bxy);
  mx = mx > mag_hi(bpx) ? mx : mag_hi(bpx);
  mx = mx > mag_hi(bpy) ? mx : mag_hi(bpy);
  mx = mx > mag_hi(bz) ? mx : mag_hi(bz);
  if (SHEAR) {
    mx = mx > mag_hi(b7) ? mx : mag_hi(b7);
    mx = mx > mag_hi(b8) ? mx : mag_hi(b8);
  }
  const int eg = (int)(mx >> 20) + kGOut;
  // unsigned arithmetic (wrapping); every final combination lies below 2^63 in magnitude
  const u64 tr = (u64)sterm(br, eg), txx = (u64)sterm(bxx, eg), tyy = (u64)sterm(byy, eg);
  const u64 txy = (u64)sterm(bxy, eg), tx = (u64)sterm(bpx, eg), ty = (u64)sterm(bpy, eg);
  const u64 tz = (u64)sterm(bz, eg);
  const u64 t7 = SHEAR ? (u64)sterm(b7, eg) : 0ull, t8 = SHEAR ? (u64)sterm(b8, eg) : 0ull;
  const u64 T = txx + tyy;
  const u64 C = 4 * tr + tz;
  const u64 X = 12 * txx - 6 * tyy + 9 * t7;  // f1, f3 part
  const u64 Y = 6 * T - X;                    // 12 yy - 6 xx - 9 p7: f2, f4 part
  const u64 a1 = C + X, a2 = C + Y;
  const u64 x12 = 12 * tx, y12 = 12 * ty;
  const u64 B = tr + 3 * T + tz;
  const u64 Q = 9 * (txy + t8);
  const u64 S = 3 * (tx + ty), D = 3 * (ty - tx);
  const u64 bq = B + Q, bm = B - Q;
  u64 n[9];
  n[1] = a1 + x12;
  n[3] = a1 - x12;
  n[2] = a2 + y12;
  n[4] = a2 - y12;
  n[5] = bq + S;
  n[7] = bq - S;
  n[6] = bm + D;
  n[8] = bm - D;
  n[0] = 4 * tr - 6 * T - 2 * tz;  // f0 / 4
  const bool bad = mx >= kFrameMaxHi;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const u64 v = round_frame_s((i64)n[k], k == 0 ? eg + 2 : eg);
    f[k] = double_of(bad ? kNaN : v);
  }
}

// The reverse mode of reduced_populations: given the adjoints mu_0..8 of the nine
// populations, the adjoints of its inputs out = {r, xx, yy, xy, px, py, zz, p7, p8}
// (the transpose of its small-integer combinations; p7, p8 only when SHEAR):
//   r  = 16 mu0 + 4 (mu1 + mu2 + mu3 + mu4) + (mu5 + mu6 + mu7 + mu8)
//   xx = -24 mu0 + 12 (mu1 + mu3) - 6 (mu2 + mu4) + 3 (mu5 + mu6 + mu7 + mu8)
//   yy = -24 mu0 - 6 (mu1 + mu3) + 12 (mu2 + mu4) + 3 (mu5 + mu6 + mu7 + mu8)
//   xy = p8 = 9 (mu5 + mu7 - mu6 - mu8)
//   px = 12 (mu1 - mu3) + 3 (mu5 - mu7 - mu6 + mu8),  py = 12 (mu2 - mu4) + 3 (mu5 - mu7 + mu6 - mu8)
//   zz = -8 mu0 + (mu1 + ... + mu8),                 p7 = 9 (mu1 + mu3 - mu2 - mu4),
// exact in one frame over the nine adjoints (coefficients summing to 72 at most:
// headroom 8) and each rounded once; p7, p8 are formed when ALL (default SHEAR) and
// are 0.0 otherwise. An adjoint out of the frames' range makes every output NaN.
constexpr int kGTr = 8;

template <bool SHEAR, bool ALL = SHEAR>
PPLBM_FX void reduced_populations_transpose(const double (&mu)[9], double (&out)[9]) {
  u64 b[9];
  unsigned mx = 0;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    b[k] = bits_of(mu[k]);
    mx = mx > mag_hi(b[k]) ? mx : mag_hi(b[k]);
  }
  const int eg = (int)(mx >> 20) + kGTr;
  u64 t[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) t[k] = (u64)sterm(b[k], eg);
  const u64 a13 = t[1] + t[3], a24 = t[2] + t[4], d13 = t[1] - t[3], d24 = t[2] - t[4];
  const u64 s57 = t[5] + t[7], s68 = t[6] + t[8], d57 = t[5] - t[7], d68 = t[6] - t[8];
  const u64 diag = s57 + s68;
  u64 n[9];
  n[0] = 16 * t[0] + 4 * (a13 + a24) + diag;
  n[1] = 3 * diag - 24 * t[0] + 12 * a13 - 6 * a24;
  n[2] = 3 * diag - 24 * t[0] - 6 * a13 + 12 * a24;
  n[3] = 9 * (s57 - s68);
  n[4] = 12 * d13 + 3 * (d57 - d68);
  n[5] = 12 * d24 + 3 * (d57 + d68);
  n[6] = a13 + a24 + diag - 8 * t[0];
  n[7] = 9 * (a13 - a24);
  n[8] = n[3];
  const bool bad = mx >= kFrameMaxHi;
  const int kout = ALL ? 9 : 7;  // ALL: p7, p8 too (the adjoints the source terms need)
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    if (k >= kout) {
      out[k] = 0.0;
      continue;
    }
    out[k] = double_of(bad ? kNaN : round_frame_s((i64)n[k], eg));
  }
}

// The reverse mode of j_h_combos: from the adjoints a1, a2, a3 of j + h, j + 2h, j + 3h,
// a4 of j - h (when MINUS) and partial adjoints j0 of j and h0 of h, the adjoints
//   jb = j0 + a1 + a2 + a3 (+ a4),  hb = h0 + a1 + 2 a2 + 3 a3 (- a4),
// exact in one frame (coefficients summing to 8 at most: headroom 5) and rounded once.
template <bool MINUS>
PPLBM_FX void j_h_combos_transpose(double a1, double a2, double a3, double a4, double j0, double h0, double* jb,
                                   double* hb) {
  const double v[6] = {a1, a2, a3, MINUS ? a4 : 0.0, j0, h0};
  u64 b[6];
  unsigned mx = 0;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    b[k] = bits_of(v[k]);
    mx = mx > mag_hi(b[k]) ? mx : mag_hi(b[k]);
  }
  const int eg = (int)(mx >> 20) + 5;
  u64 t[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) t[k] = (u64)sterm(b[k], eg);
  const u64 s = t[0] + t[1] + t[2];
  const bool bad = mx >= kFrameMaxHi;
  *jb = double_of(bad ? kNaN : round_frame_s((i64)(t[4] + s + t[3]), eg));
  *hb = double_of(bad ? kNaN : round_frame_s((i64)(t[5] + s + t[1] + 2 * t[2] - t[3]), eg));
}

// The adjoint's transpose of the Shan-Chen stencil at a node, plus the node's own
// psi adjoint: with gx_bar (sx) and gy_bar (sy) at the neighbours,
//   psi_bar = own + 4 (sxW - sxE) + 4 (syS - syN) + (sxSW + sySW) - (sxNE + syNE)
//                 + (sxNW - syNW) - (sxSE - sySE),
// exact in one frame (coefficients summing to 25: headroom 6) and rounded once. v
// holds {own, sxW, sxE, syS, syN, sxSW, sySW, sxNE, syNE, sxNW, syNW, sxSE, sySE}; a
// value out of the frames' range gives NaN.
PPLBM_FX double psi_adjoint_gather(const double (&v)[13]) {
  u64 b[13];
  unsigned mx = 0;
#pragma unroll
  for (int k = 0; k < 13; ++k) {
    b[k] = bits_of(v[k]);
    mx = mx > mag_hi(b[k]) ? mx : mag_hi(b[k]);
  }
  const int eg = (int)(mx >> 20) + 6;
  u64 t[13];
#pragma unroll
  for (int k = 0; k < 13; ++k) t[k] = (u64)sterm(b[k], eg);
  const u64 s = t[0] + 4 * ((t[1] - t[2]) + (t[3] - t[4])) + (t[5] + t[6]) - (t[7] + t[8]) + (t[9] - t[10]) -
                (t[11] - t[12]);
  return double_of(mx >= kFrameMaxHi ? kNaN : round_frame_s((i64)s, eg));
}

// The adjoint's lambda^t_i = rho_bar + c_i . j_bar (+ with SHEAR the rows 7, 8 of Eq.
// MatrixMRT times the stress moments' adjoints m7_bar, m8_bar: +-1 on the axes,
// +-1 on the diagonals), i = 1..8 (lambda_0 = rho_bar), exact in one frame
// (coefficients summing to 4: headroom 4) and each rounded once.
template <bool SHEAR>
PPLBM_FX void lambda_assembly(double rb, double jxb, double jyb, double m7b, double m8b, double (&l)[9]) {
  const double v[5] = {rb, jxb, jyb, SHEAR ? m7b : 0.0, SHEAR ? m8b : 0.0};
  u64 b[5];
  unsigned mx = 0;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    b[k] = bits_of(v[k]);
    mx = mx > mag_hi(b[k]) ? mx : mag_hi(b[k]);
  }
  const int eg = (int)(mx >> 20) + 4;
  u64 t[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) t[k] = (u64)sterm(b[k], eg);
  const u64 rp = t[0] + t[1], rm = t[0] - t[1];
  u64 n[9];
  n[1] = rp + t[3];
  n[2] = t[0] + t[2] - t[3];
  n[3] = rm + t[3];
  n[4] = t[0] - t[2] - t[3];
  n[5] = rp + t[2] + t[4];
  n[6] = rm + t[2] - t[4];
  n[7] = rm - t[2] + t[4];
  n[8] = rp - t[2] - t[4];
  const bool bad = mx >= kFrameMaxHi;
  l[0] = rb;
#pragma unroll
  for (int k = 1; k < 9; ++k) l[k] = double_of(bad ? kNaN : round_frame_s((i64)n[k], eg));
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
