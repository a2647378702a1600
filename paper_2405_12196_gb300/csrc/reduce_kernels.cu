// Scalar product of two tensors on the same legs, in FP64: the sum over the
// elements of their common blocks of A's element times B's. The paper leaves the
// scalar reductions of a tensor network (norms, overlaps, expectation values) to
// its backend; here they stay in FP64 beside the contraction kernels.
//
// Deterministic: the planner fixes each CTA's share (consecutive runs of common
// elements, at most 8192); a thread sums a fixed subset of them with four
// interleaved accumulators, a CTA combines its threads in a fixed tree and writes
// one partial, and one CTA adds the partials in a fixed order. Repeated calls give
// identical bits. HBM-bound: 16 bytes read per common element.
#include <cuda_runtime.h>

#include "kernels.hpp"

namespace ytn {

namespace {

constexpr int kThreads = 256;
constexpr int kFinalThreads = 1024;

__device__ __forceinline__ double block_sum(double v, double *ws) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) ws[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += ws[w];
  return t;
}

__global__ void __launch_bounds__(kThreads) vdot_partial_kernel(const VdotChunk *__restrict__ chunks,
                                                                const VdotPiece *__restrict__ pieces,
                                                                const double *a, const double *b,
                                                                double *__restrict__ partials) {
  __shared__ double ws[kThreads / 32];
  const VdotChunk ch = chunks[blockIdx.x];
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  for (int k = ch.first; k < ch.first + ch.count; k++) {
    const VdotPiece pc = pieces[k];
    const double *pa = a + pc.a_off, *pb = b + pc.b_off;
    int e = threadIdx.x;
    for (; e + 3 * kThreads < pc.len; e += 4 * kThreads) {
      const double a0 = pa[e], a1 = pa[e + kThreads], a2 = pa[e + 2 * kThreads], a3 = pa[e + 3 * kThreads];
      const double b0 = pb[e], b1 = pb[e + kThreads], b2 = pb[e + 2 * kThreads], b3 = pb[e + 3 * kThreads];
      s0 = fma(a0, b0, s0);
      s1 = fma(a1, b1, s1);
      s2 = fma(a2, b2, s2);
      s3 = fma(a3, b3, s3);
    }
    for (; e < pc.len; e += kThreads) s0 = fma(pa[e], pb[e], s0);
  }
  const double t = block_sum((s0 + s1) + (s2 + s3), ws);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kFinalThreads) vdot_final_kernel(const double *__restrict__ partials, int n,
                                                                   double *out) {
  __shared__ double ws[kFinalThreads / 32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += kFinalThreads) s += partials[i];
  const double t = block_sum(s, ws);
  if (threadIdx.x == 0) out[0] = t;
}

}  // namespace

cudaError_t launch_vdot(const VdotChunk *chunks, int64_t nchunks, const VdotPiece *pieces, const double *a,
                        const double *b, double *partials, double *out, cudaStream_t stream) {
  if (nchunks > INT32_MAX) return cudaErrorInvalidValue;
  if (nchunks > 0) vdot_partial_kernel<<<(unsigned)nchunks, kThreads, 0, stream>>>(chunks, pieces, a, b, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  vdot_final_kernel<<<1, kFinalThreads, 0, stream>>>(partials, (int)nchunks, out);
  return cudaGetLastError();
}

}  // namespace ytn
