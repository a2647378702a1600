// Split of FP64 sector matrices into BF16 slices for the split-precision grouped
// GEMM (an error-free splitting in the manner of Ozaki, Ogita, Oishi and Rump,
// Numer. Algorithms 2012, with power-of-two scales per row).
//
// For a row x_r of an operand (a row of A_q, or a column of B_q), with
// e_r = 2 + floor(log2 max_k |x_rk|) (one bit of headroom: |x_rk| < 2^(e_r - 1)),
// every element is rounded to the integer u = round(x_rk 2^(8s - e_r)),
// |u| <= 2^(8s-1), and u is written in balanced base 256 (s = slices in use, <= 6):
//     u = sum_{p=0..s-1} d_p 256^(s-1-p),  d_p in [-128, 127] for p >= 1,
//     d_0 in [-128, 128],
// so x_rk = 2^e_r (sum_p d_p 2^{-8(p+1)} + t) with |t| <= 2^(-8s-1). Slices beyond
// s are zero. Slice p holds d_p 2^{-8p}: a signed integer of magnitude at most 2^7
// times a power of two, exact in BF16; products of two slices are exact in FP32
// and at most 2^14 times their power of two, which lets the GEMM sum 256 of K
// exactly per accumulator. The digits are taken from the FP64 bit pattern with
// integer operations only (no FP64 arithmetic, which is slow on this GPU). Zero
// and subnormal inputs give zero digits.
//
// Output layout: for operand block (row tile rt, K stage kt) six consecutive
// 128 x 32 BF16 slices, each K-major with the 64-byte swizzle (16-byte chunk c of
// row r stored at chunk position c ^ ((r >> 1) & 3)), the layout the tensor
// cores read from shared memory; rows and K beyond the operand are zero.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "kernels.hpp"
#include "split_digits.cuh"

namespace ytn {

namespace {

// Row exponents: e_r = maxE - 1021 over the row (maxE = largest biased exponent,
// 0 for a zero row). An item covers 128 rows and up to 256 of K; its per-row
// maxima are combined into E with atomicMax (exact and order-independent), E
// having been set below every exponent beforehand. Rows past the operand are
// left alone (no kernel reads them). The item's largest exponent also goes into
// emax[op], the operand's largest (the reference scale of the accuracy check).
__global__ void __launch_bounds__(256) split_exp_kernel(const SplitOperand *__restrict__ ops,
                                                        const SplitItem *__restrict__ items,
                                                        const double *__restrict__ wa,
                                                        const double *__restrict__ wb,
                                                        int32_t *__restrict__ ea, int32_t *__restrict__ eb,
                                                        int32_t *__restrict__ emax) {
  const SplitItem it = items[blockIdx.x];
  const SplitOperand o = ops[it.op];
  const bool isA = (it.op & 1) == 0;
  const double *X = (isA ? wa : wb) + o.src_off;
  int32_t *E = (isA ? ea : eb) + o.exp_off;
  const int r0 = it.rt * kSplitBM;
  const int k_lo = it.kt0 * kSplitBK, k_hi = min(o.K, (it.kt0 + it.nkt) * kSplitBK);
  __shared__ int red[2][kSplitBM];
  __shared__ int wmax[8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int mine = 0;   // largest biased exponent this thread saw
  if (o.kmajor) {
    // rows of K contiguous elements: one warp per row
    for (int rr = warp; rr < kSplitBM; rr += 8) {
      const int r = r0 + rr;
      if (r >= o.rows) break;   // uniform in the warp
      const double *row = X + (int64_t)r * o.K;
      int m = 0;
#pragma unroll 8
      for (int k = k_lo + lane; k < k_hi; k += 32) m = max(m, biased_exp(__ldg(row + k)));
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, s));
      if (lane == 0) atomicMax(E + r, m - 1021);
      mine = max(mine, m);
    }
  } else {
    // K rows of `rows` contiguous elements: thread per row, two halves of the K range
    const int rr = tid & (kSplitBM - 1), half = tid >> 7;
    const int r = r0 + rr;
    int m = 0;
    if (r < o.rows)
#pragma unroll 4
      for (int k = k_lo + half; k < k_hi; k += 2) m = max(m, biased_exp(__ldg(X + (int64_t)k * o.rows + r)));
    red[half][rr] = m;
    mine = m;
    __syncthreads();
    if (tid < kSplitBM && r0 + tid < o.rows) atomicMax(E + r0 + tid, max(red[0][tid], red[1][tid]) - 1021);
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) mine = max(mine, __shfl_xor_sync(0xffffffffu, mine, s));
  if (lane == 0) wmax[warp] = mine;
  __syncthreads();
  if (tid == 0) {
    int m = wmax[0];
#pragma unroll
    for (int w = 1; w < 8; w++) m = max(m, wmax[w]);
    atomicMax(emax + it.op, m - 1021);
  }
}

// Slices: one 128 x 32 stage at a time through shared memory (raw FP64 bits).
__global__ void __launch_bounds__(256, 6) split_slice_kernel(const SplitOperand *__restrict__ ops,
                                                          const SplitItem *__restrict__ items,
                                                          const double *__restrict__ wa,
                                                          const double *__restrict__ wb,
                                                          const int32_t *__restrict__ ea,
                                                          const int32_t *__restrict__ eb,
                                                          uint8_t *__restrict__ sa, uint8_t *__restrict__ sb,
                                                          int s) {
  __shared__ unsigned long long tile[kSplitBM][kSplitBK + 1];
  __shared__ int rexp[kSplitBM];
  const SplitItem it = items[blockIdx.x];
  const SplitOperand o = ops[it.op];
  const bool isA = (it.op & 1) == 0;
  const double *X = (isA ? wa : wb) + o.src_off;
  const int32_t *E = (isA ? ea : eb) + o.exp_off;
  uint8_t *S = (isA ? sa : sb) + o.slice_off;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r0 = it.rt * kSplitBM;
  if (tid < kSplitBM) rexp[tid] = r0 + tid < o.rows ? E[r0 + tid] : -1021;
  for (int kt = it.kt0; kt < it.kt0 + it.nkt; kt++) {
    const int k0 = kt * kSplitBK;
    __syncthreads();
    if (o.kmajor) {
      for (int rr = warp; rr < kSplitBM; rr += 8) {
        const int r = r0 + rr, k = k0 + lane;
        double v = 0.0;
        if (r < o.rows && k < o.K) v = __ldg(X + (int64_t)r * o.K + k);
        tile[rr][lane] = (unsigned long long)__double_as_longlong(v);
      }
    } else {
      for (int kk = warp; kk < kSplitBK; kk += 8) {
        const int k = k0 + kk;
#pragma unroll
        for (int q = 0; q < kSplitBM / 32; q++) {
          const int rr = q * 32 + lane, r = r0 + rr;
          double v = 0.0;
          if (r < o.rows && k < o.K) v = __ldg(X + (int64_t)k * o.rows + r);
          tile[rr][kk] = (unsigned long long)__double_as_longlong(v);
        }
      }
    }
    __syncthreads();
    uint8_t *blk = S + ((int64_t)it.rt * o.ks + kt) * kBlockBytes;
    // 128 rows x 4 chunks of 8 elements; two chunks per thread
    for (int task = tid; task < kSplitBM * 4; task += 256) {
      const int rr = task >> 2, c = task & 3;
      uint32_t packed[kSlices][4];
      slice_digits8(&tile[rr][c * 8], rexp[rr], s, packed);
      store_slices(blk, slice_pos(rr, c), s, packed);
    }
  }
}

}  // namespace

cudaError_t launch_split_prep(const SplitOperand *ops, const SplitItem *exp_items, int64_t nexp,
                              const SplitItem *slice_items, int64_t nslice, const double *wa, const double *wb,
                              int32_t *ea, int32_t *eb, int32_t *emax, uint8_t *sa, uint8_t *sb, int slices,
                              cudaStream_t stream) {
  if (nexp > INT32_MAX || nslice > INT32_MAX || slices < 1 || slices > kSlices) return cudaErrorInvalidValue;
  if (nexp > 0) split_exp_kernel<<<(unsigned)nexp, 256, 0, stream>>>(ops, exp_items, wa, wb, ea, eb, emax);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (nslice > 0) split_slice_kernel<<<(unsigned)nslice, 256, 0, stream>>>(ops, slice_items, wa, wb, ea, eb, sa, sb, slices);
  return cudaGetLastError();
}

}  // namespace ytn
