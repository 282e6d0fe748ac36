// Accuracy self-test of the FP64 reciprocal and square root used by the step
// kernels (fp64.cuh) against CUDA's correctly rounded 1/x and sqrt(x).
#include <cuda_runtime.h>

#include "../../include/pplbm.h"
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
