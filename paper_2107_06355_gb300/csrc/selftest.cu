// Accuracy self-test of the FP64 reciprocal and square root used by the step
// kernels (fp64.cuh) against CUDA's correctly rounded 1/x and sqrt(x).
#include <cuda_runtime.h>

#include "../../include/pplbm.h"
#include "fixsum.cuh"
#include "fp64.cuh"

namespace pplbm {
namespace {

// splitmix64 (Steele, Lea, Flood 2014): a counter-based 64-bit mixer
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_fp64_selftest(long long n, unsigned long long seed, unsigned long long* out) {
  double er = 0.0, es = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long h = splitmix64(seed ^ (unsigned long long)i);
    // x = m * 2^k, m in [1, 2), k in [-60, 60]: covers the densities, psi^2 and (1 - eta)^3 met in the step
    const double m = 1.0 + (double)(h >> 11) * 0x1.0p-53;
    const int k = (int)((h & 0x7Full) % 121) - 60;
    const double x = ldexp(m, k);
    const double r = fast_rcp(x), rr = 1.0 / x;
    const double s = fast_sqrt(x), ss = sqrt(x);
    er = fmax(er, fabs(r - rr) / rr);
    es = fmax(es, fabs(s - ss) / ss);
  }
  atomicMax(&out[0], (unsigned long long)__double_as_longlong(er));
  atomicMax(&out[1], (unsigned long long)__double_as_longlong(es));
}

// add_pos_int and add_int against the FP64 pipe's x + y, bit for bit. Four kinds of
// pairs: independent exponents around 1; exponent gaps 0..63; low bits of the smaller
// operand forced to a half-way pattern (ties, both parities); the larger operand's
// significand all ones (rounding carries into the exponent). add_int also sees every
// sign combination, signed zeros, and, in the last kind, operands 0..7 ulp apart
// (exact and near cancellation).
__global__ void k_int_add_selftest(long long n, unsigned long long seed, unsigned long long* out) {
  typedef unsigned long long u64;
  const u64 M = (1ull << 52) - 1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const u64 h = splitmix64(seed ^ (u64)i), g = splitmix64(h);
    const int kind = (int)(h & 3);
    const u64 ea = 1023 - 40 + ((h >> 2) & 63);
    u64 eb = 1023 - 40 + ((g >> 2) & 63);
    u64 ma = (h >> 8) & M, mb = (g >> 8) & M;
    if (kind == 1 || kind == 2) eb = ea - ((g >> 58) & 63);
    if (kind == 2) {
      const int d = (int)(ea - eb);
      if (d >= 1 && d <= 52) mb = (mb & ~((1ull << d) - 1)) | (1ull << (d - 1));  // half an ulp of a, exactly
    }
    if (kind == 3) ma = M;
    const u64 a = (ea << 52) | ma, b = (eb << 52) | mb;
    const double x = __longlong_as_double((long long)a), y = __longlong_as_double((long long)b);
    const u64 want = (u64)__double_as_longlong(x + y);
    const u64 got = (u64)__double_as_longlong(add_pos_int(x, y));
    if (got != want && atomicAdd(&out[0], 1ull) == 0ull) {
      out[1] = a;
      out[2] = b;
      out[3] = got;
      out[4] = want;
    }
    // add_int on the same magnitudes with every sign combination, and on a pair that
    // cancels exactly or up to the last bits (x + (-x), x + (-(x + k ulp)))
    const u64 sa = (g >> 60) & 1, sb = (g >> 61) & 1;
    u64 b2 = (kind == 3 ? (a + ((g >> 56) & 7)) : b) | (sb << 63);
    if (((g >> 62) & 3) == 3) b2 = sb << 63;   // a zero of either sign
    const u64 a2 = a | (sa << 63);
    const double x2 = __longlong_as_double((long long)a2), y2 = __longlong_as_double((long long)b2);
    const u64 want2 = (u64)__double_as_longlong(x2 + y2);
    const u64 got2 = (u64)__double_as_longlong(add_int(x2, y2));
    // and the subtraction x2 - (-y2), the same sum through sub_int
    const u64 got3 = (u64)__double_as_longlong(sub_int(x2, -y2));
    if (got3 != want2 && atomicAdd(&out[0], 1ull) == 0ull) {
      out[1] = a2;
      out[2] = b2 ^ (1ull << 63);
      out[3] = got3;
      out[4] = want2;
    }
    if (got2 != want2 && atomicAdd(&out[0], 1ull) == 0ull) {
      out[1] = a2;
      out[2] = b2;
      out[3] = got2;
      out[4] = want2;
    }
  }
}

}  // namespace
}  // namespace pplbm

extern "C" pplbm_status pplbm_fp64_selftest(long long n, unsigned long long seed, double* out, void* stream) {
  if (n < 1 || !out) return PPLBM_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(out, 0, 2 * sizeof(double), s) != cudaSuccess) return PPLBM_ERR_CUDA;
  pplbm::k_fp64_selftest<<<304, 256, 0, s>>>(n, seed, (unsigned long long*)out);
  if (cudaGetLastError() != cudaSuccess) return PPLBM_ERR_CUDA;
  return PPLBM_OK;
}

// FP64 issue-rate probe: every thread runs CH independent chains of one FP64
// operation (OP 0: x <- x * b + c, 1: x <- x + c, 2: x <- x * b; |b| < 1 keeps the
// chains bounded), so the FP64 pipe is the only limit; OP 3 runs chains of the
// integer-pipe addition add_pos_int instead (y <- y + c), and OP 4 both, one FMA and
// one integer-pipe addition per chain and round (whether the two pipes overlap); OP 5
// chains of 64-bit integer to double conversions, OP 6 of double to 64-bit integer
// conversions (each with one integer operation feeding the result back). The sum of
// the chains goes to `sink` so that none of the work is dead.
namespace pplbm {
namespace {

constexpr int kPeakThreads = 256;

template <int CH, int OP>
__global__ void __launch_bounds__(kPeakThreads) k_fp64_peak(long long iters, double b, double c, double* sink) {
  double x[CH], y[CH];
  unsigned long long z[CH];
#pragma unroll
  for (int k = 0; k < CH; ++k) {
    x[k] = (double)(threadIdx.x + k) * 1e-3;
    y[k] = 1.0 + x[k];
    z[k] = 1000ull + threadIdx.x + k;
  }
  if (OP == 6) {
#pragma unroll
    for (int k = 0; k < CH; ++k) x[k] = 1e6 + x[k];  // values in [1e6, 1e6 + 1): conversions stay in range
  }
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < CH; ++k) {
      if (OP == 0 || OP == 4) x[k] = fma(x[k], b, c);
      if (OP == 1) x[k] = x[k] + c;
      if (OP == 2) x[k] = x[k] * b;
      if (OP == 3 || OP == 4) y[k] = add_pos_int(y[k], c);
      if (OP == 5) z[k] += (unsigned long long)__double_as_longlong(__ll2double_rn((long long)z[k]));
      if (OP == 6) x[k] = __longlong_as_double(__double_as_longlong(x[k]) ^ (__double2ll_rz(x[k]) & 1ll));
    }
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < CH; ++k) s += x[k] + y[k] + (double)(z[k] & 1ull);
  if (s == 12345.678) sink[0] = s;  // never true for these chains; keeps them live
}

template <int OP>
bool launch_peak(int chains, int blocks, long long iters, double* sink, cudaStream_t s) {
  switch (chains) {
    case 1: k_fp64_peak<1, OP><<<blocks, kPeakThreads, 0, s>>>(iters, 0.999999, 1e-7, sink); return true;
    case 2: k_fp64_peak<2, OP><<<blocks, kPeakThreads, 0, s>>>(iters, 0.999999, 1e-7, sink); return true;
    case 4: k_fp64_peak<4, OP><<<blocks, kPeakThreads, 0, s>>>(iters, 0.999999, 1e-7, sink); return true;
    case 8: k_fp64_peak<8, OP><<<blocks, kPeakThreads, 0, s>>>(iters, 0.999999, 1e-7, sink); return true;
    case 16: k_fp64_peak<16, OP><<<blocks, kPeakThreads, 0, s>>>(iters, 0.999999, 1e-7, sink); return true;
    case 32: k_fp64_peak<32, OP><<<blocks, kPeakThreads, 0, s>>>(iters, 0.999999, 1e-7, sink); return true;
  }
  return false;
}

}  // namespace
}  // namespace pplbm

extern "C" pplbm_status pplbm_fp64_peak(int32_t blocks_per_sm, int32_t chains, int32_t op, long long iters,
                                        double* sink, double* out, void* stream) {
  if (blocks_per_sm < 1 || blocks_per_sm > 64 || iters < 1 || !sink || !out || op < 0 || op > 6 ||
      !(chains == 1 || chains == 2 || chains == 4 || chains == 8 || chains == 16 || chains == 32))
    return PPLBM_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PPLBM_ERR_CUDA;
  const int blocks = sms * blocks_per_sm;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return PPLBM_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return PPLBM_ERR_CUDA;
  }
  pplbm_status st = PPLBM_OK;
  float ms = 0.f;
  cudaEventRecord(e0, s);
  if (op == 0) pplbm::launch_peak<0>(chains, blocks, iters, sink, s);
  else if (op == 1) pplbm::launch_peak<1>(chains, blocks, iters, sink, s);
  else if (op == 2) pplbm::launch_peak<2>(chains, blocks, iters, sink, s);
  else if (op == 3) pplbm::launch_peak<3>(chains, blocks, iters, sink, s);
  else if (op == 4) pplbm::launch_peak<4>(chains, blocks, iters, sink, s);
  else if (op == 5) pplbm::launch_peak<5>(chains, blocks, iters, sink, s);
  else pplbm::launch_peak<6>(chains, blocks, iters, sink, s);
  cudaEventRecord(e1, s);
  if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
      cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f))
    st = PPLBM_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != PPLBM_OK) return st;
  const double instr = (double)blocks * pplbm::kPeakThreads * (double)iters * chains;
  out[0] = instr / (ms * 1e-3);  // FP64 instructions (op 3: integer-pipe additions) per thread per second
  out[1] = ms;
  out[2] = (double)blocks;
  return PPLBM_OK;
}

extern "C" pplbm_status pplbm_int_add_selftest(long long n, unsigned long long seed, unsigned long long* out,
                                               void* stream) {
  if (n < 1 || !out) return PPLBM_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(out, 0, 5 * sizeof(unsigned long long), s) != cudaSuccess) return PPLBM_ERR_CUDA;
  pplbm::k_int_add_selftest<<<1216, 256, 0, s>>>(n, seed, out);
  if (cudaGetLastError() != cudaSuccess) return PPLBM_ERR_CUDA;
  return PPLBM_OK;
}

// The fixed-point sums of fixsum.cuh on caller data, one thread per row.
namespace pplbm {
namespace {

__global__ void k_fixsum_eval(long long n, const double* f, const double* p, double* out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) v[k] = f[9 * i + k];
  double* o = out + 8 * i;
  unsigned mx = 0;
  double r[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const bool ok = fx::positive_normal_range(v, &mx);
  if (ok) fx::density_moments<true>(v, fx::frame_top(mx), &r[0], &r[1], &r[2], &r[3], &r[4]);
#pragma unroll
  for (int k = 0; k < 5; ++k) o[k] = r[k];
  o[5] = ok ? 1.0 : 0.0;
  const double* q = p + 8 * i;
  fx::shan_chen_stencil(q[0], q[1], q[2], q[3], q[4], q[5], q[6], q[7], &o[6], &o[7]);
}

}  // namespace
}  // namespace pplbm

extern "C" pplbm_status pplbm_fixsum_eval(long long n, const double* f, const double* p, double* out, void* stream) {
  if (n < 0 || n > 0x7FFFFFFFLL * 255 || (n > 0 && (!f || !p || !out))) return PPLBM_ERR_ARG;
  if (n == 0) return PPLBM_OK;
  pplbm::k_fixsum_eval<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n, f, p, out);
  return cudaGetLastError() == cudaSuccess ? PPLBM_OK : PPLBM_ERR_CUDA;
}

// The collision pass's fixed-point output stage and sums on caller data, one thread per row.
namespace pplbm {
namespace {

template <bool SHEAR>
__global__ void k_fixsum_collision_eval(long long n, const double* q, const double* jh, double* out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* r = q + 9 * i;
  double f[9];
  fx::reduced_populations<SHEAR>(r[0], r[1], r[2], r[3], r[4], r[5], r[6], SHEAR ? r[7] : 0.0, SHEAR ? r[8] : 0.0, f);
  double* o = out + 13 * i;
#pragma unroll
  for (int k = 0; k < 9; ++k) o[k] = f[k];
  fx::j_h_combos<true>(jh[2 * i], jh[2 * i + 1], &o[9], &o[10], &o[11], &o[12]);
}

}  // namespace
}  // namespace pplbm

extern "C" pplbm_status pplbm_fixsum_collision_eval(long long n, int32_t shear, const double* q, const double* jh,
                                                    double* out, void* stream) {
  if (n < 0 || n > 0x7FFFFFFFLL * 255 || (n > 0 && (!q || !jh || !out))) return PPLBM_ERR_ARG;
  if (n == 0) return PPLBM_OK;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  cudaStream_t s = (cudaStream_t)stream;
  if (shear)
    pplbm::k_fixsum_collision_eval<true><<<blocks, 256, 0, s>>>(n, q, jh, out);
  else
    pplbm::k_fixsum_collision_eval<false><<<blocks, 256, 0, s>>>(n, q, jh, out);
  return cudaGetLastError() == cudaSuccess ? PPLBM_OK : PPLBM_ERR_CUDA;
}

// The reverse-mode stages on caller data, one thread per row.
namespace pplbm {
namespace {

template <bool SHEAR>
__global__ void k_fixsum_adjoint_eval(long long n, const double* mu, const double* a, const double* gth,
                                      const double* lam, double* out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double m[9], u[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) m[k] = mu[9 * i + k];
  fx::reduced_populations_transpose<SHEAR>(m, u);
  double* o = out + 21 * i;
#pragma unroll
  for (int k = 0; k < 9; ++k) o[k] = u[k];
  const double* q = a + 6 * i;
  fx::j_h_combos_transpose<true>(q[0], q[1], q[2], q[3], q[4], q[5], &o[9], &o[10]);
  double gv[13];
#pragma unroll
  for (int k = 0; k < 13; ++k) gv[k] = gth[13 * i + k];
  o[11] = fx::psi_adjoint_gather(gv);
  const double* r = lam + 5 * i;
  double l[9];
  fx::lambda_assembly<SHEAR>(r[0], r[1], r[2], r[3], r[4], l);
#pragma unroll
  for (int k = 0; k < 9; ++k) o[12 + k] = l[k];
}

}  // namespace
}  // namespace pplbm

extern "C" pplbm_status pplbm_fixsum_adjoint_eval(long long n, int32_t shear, const double* mu, const double* a,
                                                  const double* gth, const double* lam, double* out, void* stream) {
  if (n < 0 || n > 0x7FFFFFFFLL * 255 || (n > 0 && (!mu || !a || !gth || !lam || !out))) return PPLBM_ERR_ARG;
  if (n == 0) return PPLBM_OK;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  cudaStream_t s = (cudaStream_t)stream;
  if (shear)
    pplbm::k_fixsum_adjoint_eval<true><<<blocks, 256, 0, s>>>(n, mu, a, gth, lam, out);
  else
    pplbm::k_fixsum_adjoint_eval<false><<<blocks, 256, 0, s>>>(n, mu, a, gth, lam, out);
  return cudaGetLastError() == cudaSuccess ? PPLBM_OK : PPLBM_ERR_CUDA;
}
