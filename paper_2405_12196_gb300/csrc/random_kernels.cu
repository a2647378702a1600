// N(0, 1) data for random tensors (the paper's rand, Sec. II.A): Philox4x32-10
// (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3",
// SC'11), a counter-based generator, so every element is a pure function of the
// seed and its index; pairs of words become normals by the Box-Muller transform.
#include <cuda_runtime.h>

#include "kernels.hpp"

namespace ytn {

namespace {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; r++) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// One thread per group of four elements: element i = 4q + j takes word j of the
// generator at counter (q low, q high, 0, 0).
__global__ void __launch_bounds__(256) fill_normal_kernel(uint2 key, int64_t n, double *__restrict__ out) {
  const int64_t ngroups = (n + 3) / 4;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < ngroups; q += (int64_t)gridDim.x * blockDim.x) {
    const uint4 w = philox4x32_10(make_uint4((uint32_t)q, (uint32_t)(q >> 32), 0u, 0u), key);
    const uint32_t x[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const double u = ((double)x[2 * h] + 1.0) * 2.3283064365386963e-10;   // 2^-32
      const double v = (double)x[2 * h + 1] * 2.3283064365386963e-10;
      const double r = sqrt(-2.0 * log(u));
      double sn, cs;
      sincospi(2.0 * v, &sn, &cs);
      const int64_t i = 4 * q + 2 * h;
      if (i < n) out[i] = r * cs;
      if (i + 1 < n) out[i + 1] = r * sn;
    }
  }
}

}  // namespace

cudaError_t launch_fill_normal(uint64_t seed, int64_t n, double *out, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int64_t groups = (n + 3) / 4;
  const unsigned grid = (unsigned)std::min<int64_t>((groups + 255) / 256, 152 * 16);
  fill_normal_kernel<<<grid, 256, 0, stream>>>(make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)), n, out);
  return cudaGetLastError();
}

}  // namespace ytn
