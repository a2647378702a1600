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

// CPLX: the pieces run over interleaved (re, im) doubles, and <A, B> = sum conj(a) b:
// re = sum over all doubles of a b; im = sum over pairs of a_re b_im - a_im b_re.
template <bool CPLX>
__global__ void __launch_bounds__(kThreads) vdot_partial_kernel(const VdotChunk *__restrict__ chunks,
                                                                const VdotPiece *__restrict__ pieces,
                                                                const double *a, const double *b,
                                                                double *__restrict__ partials) {
  __shared__ double ws[kThreads / 32];
  const VdotChunk ch = chunks[blockIdx.x];
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0, t0 = 0.0, t1 = 0.0;
  for (int k = ch.first; k < ch.first + ch.count; k++) {
    const VdotPiece pc = pieces[k];
    const double *pa = a + pc.a_off, *pb = b + pc.b_off;
    int e = threadIdx.x;
    if (!CPLX) {
      for (; e + 3 * kThreads < pc.len; e += 4 * kThreads) {
        const double a0 = pa[e], a1 = pa[e + kThreads], a2 = pa[e + 2 * kThreads], a3 = pa[e + 3 * kThreads];
        const double b0 = pb[e], b1 = pb[e + kThreads], b2 = pb[e + 2 * kThreads], b3 = pb[e + 3 * kThreads];
        s0 = fma(a0, b0, s0);
        s1 = fma(a1, b1, s1);
        s2 = fma(a2, b2, s2);
        s3 = fma(a3, b3, s3);
      }
      for (; e < pc.len; e += kThreads) s0 = fma(pa[e], pb[e], s0);
    } else {
      // thread e takes one double; its pair's other half comes from the same cache line
      for (; e < pc.len; e += kThreads) {
        const double x = pa[e], y = pb[e], z = pb[e ^ 1];
        s0 = fma(x, y, s0);
        if (e & 1) t1 = fma(x, z, t1);   // a_im b_re
        else t0 = fma(x, z, t0);         // a_re b_im
      }
    }
  }
  const double t = block_sum((s0 + s1) + (s2 + s3), ws);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
  if (CPLX) {
    __syncthreads();
    const double u = block_sum(t0 - t1, ws);
    if (threadIdx.x == 0) partials[gridDim.x + blockIdx.x] = u;
  }
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
                        const double *b, double *partials, double *out, bool complex_data, cudaStream_t stream) {
  if (nchunks > INT32_MAX / 2) return cudaErrorInvalidValue;
  if (nchunks > 0) {
    if (complex_data)
      vdot_partial_kernel<true><<<(unsigned)nchunks, kThreads, 0, stream>>>(chunks, pieces, a, b, partials);
    else
      vdot_partial_kernel<false><<<(unsigned)nchunks, kThreads, 0, stream>>>(chunks, pieces, a, b, partials);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  vdot_final_kernel<<<1, kFinalThreads, 0, stream>>>(partials, (int)nchunks, out);
  if (complex_data) vdot_final_kernel<<<1, kFinalThreads, 0, stream>>>(partials + nchunks, (int)nchunks, out + 1);
  return cudaGetLastError();
}

}  // namespace ytn
