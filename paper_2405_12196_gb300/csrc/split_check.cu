// Accuracy check of the split-precision products, with its FP64 fallback.
//
// The split GEMM rounds each operand row (a row of A_q, a column of B_q) to the
// digits kept at its power-of-two scale 2^e, drops the digit products of order
// >= s and rounds the FP32 accumulator of the orders >= 3. Every one of these
// errors is a small multiple of the product of the two scales, 2^(e_i + f_j),
// per element of C_q, and grows like sqrt(K) over the contraction (independent
// roundings). So the absolute error of C_q is estimated, per element, by
// eta sqrt(K) 2^(e_i + f_j), and its relative Frobenius error by
//     est_q = eta sqrt(K_q sum_i 4^(e_i) sum_j 4^(f_j)) / ||C_q||_F,
// which sees the data through the scales and the result: when a row holds one
// large element and the rest far below it, or when the products cancel, the
// scales are large against |c_ij| and the estimate grows with that ratio.
//
// One CTA per sector computes est_q from the exponents and the ||C_q||^2 that
// the GEMM epilogue summed (both taken relative to the operands' largest
// exponents, so nothing overflows). The last CTA to finish:
//   - lists the sectors with est_q > rtol, in sector order, with the running
//     counts of their 64 x 64 tiles and of their gather work items (the FP64
//     recomputation reads these lists);
//   - writes the call's record: the relative error of the whole result before
//     and after the fallback (sectors weighted by their norms), the largest
//     per-sector estimate, the number of recomputed sectors and their FLOPs;
//   - raises the tolerance flag in the context's status word when even the
//     result after the fallback is estimated above rtol.
// Everything runs on the device, so a call stays asynchronous and can be
// recorded into a graph.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>

#include "kernels.hpp"

namespace ytn {

namespace {

constexpr int kThreads = 256;

// 4^k for k <= 0 as an FP64 value built from its bits (0 below the normal range).
__device__ __forceinline__ double pow4(int k) {
  return k >= -511 ? __longlong_as_double((long long)(1023 + 2 * k) << 52) : 0.0;
}

__device__ __forceinline__ double block_sum(double v, double *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < kThreads / 32; w++) t += red[w];
  return t;
}

__device__ __forceinline__ int block_max(int v, int *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  int t = red[0];
#pragma unroll
  for (int w = 1; w < kThreads / 32; w++) t = max(t, red[w]);
  return t;
}

// Exclusive prefix sum over the block (one value per thread); returns the
// thread's offset and the block total in *total.
__device__ __forceinline__ int block_scan(int v, int *red, int *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  __syncthreads();
  if (lane == 31) red[warp] = x;
  __syncthreads();
  int before = 0, all = 0;
#pragma unroll
  for (int w = 0; w < kThreads / 32; w++) {
    if (w < warp) before += red[w];
    all += red[w];
  }
  *total = all;
  return before + x - v;
}

// A zero operand (every exponent at the zero-row value) gives an exact zero product.
constexpr int kZeroExp = -1021;

__global__ void __launch_bounds__(kThreads) split_check_kernel(
    const SplitSector *__restrict__ sectors, int nsec, const int32_t *__restrict__ ea, const int32_t *__restrict__ eb,
    const int32_t *__restrict__ emax, const float *__restrict__ normsq, double *__restrict__ secv,
    int32_t *__restrict__ flagged, int32_t *__restrict__ tile_end, int32_t *__restrict__ item_end_a,
    int32_t *__restrict__ item_end_b, SplitRecord *rec, double eta_split, double eta_fp64, double rtol, int slices,
    int *status) {
  __shared__ double dred[kThreads / 32];
  __shared__ int ired[kThreads / 32];
  __shared__ int is_last;
  const int q = blockIdx.x, tid = threadIdx.x;
  const SplitSector sc = sectors[q];
  const int EA = emax[2 * q], EB = emax[2 * q + 1];
  const bool zero = EA <= kZeroExp || EB <= kZeroExp || sc.M == 0 || sc.N == 0 || sc.K == 0;
  double se = 0.0, sf = 0.0;
  if (!zero) {
    for (int i = tid; i < sc.M; i += kThreads) se += pow4(ea[sc.ea_off + i] - EA);
    for (int j = tid; j < sc.N; j += kThreads) sf += pow4(eb[sc.eb_off + j] - EB);
  }
  se = block_sum(se, dred);
  sf = block_sum(sf, dred);
  if (tid == 0) secv[q] = zero ? 0.0 : (double)sc.K * se * sf;
  // the last CTA to get here sees every sector's value
  __threadfence();
  __syncthreads();
  if (tid == 0) is_last = atomicAdd(&rec->done_blocks, 1) == nsec - 1;
  __syncthreads();
  if (!is_last) return;
  __threadfence();

  // reference exponent: the largest emax_A + emax_B among sectors with data
  int g = INT_MIN;
  for (int s = tid; s < nsec; s += kThreads)
    if (__ldcg(secv + s) > 0.0 || normsq[s] > 0.0f) g = max(g, emax[2 * s] + emax[2 * s + 1]);
  g = block_max(g, ired);
  double norm = 0.0, err_split = 0.0, err_after = 0.0, flops = 0.0, worst = 0.0;
  int nflag = 0, ntile = 0, nia = 0, nib = 0;
  for (int base = 0; base < nsec; base += kThreads) {
    const int s = base + tid;
    int flag = 0, tiles = 0, ia = 0, ib = 0;
    if (s < nsec) {
      const double v = __ldcg(secv + s), n2 = (double)normsq[s];
      double est = 0.0;
      if (v > 0.0) est = n2 > 0.0 ? eta_split * sqrt(v / n2) : INFINITY;
      flag = est > rtol;
      worst = fmax(worst, est);
      if (g != INT_MIN) {
        const double w = pow4(emax[2 * s] + emax[2 * s + 1] - g);
        norm += n2 * w;
        err_split += eta_split * eta_split * v * w;
        err_after += (flag ? eta_fp64 * eta_fp64 : eta_split * eta_split) * v * w;
      }
      if (flag) {
        const SplitSector t = sectors[s];
        tiles = ((t.M + 63) / 64) * ((t.N + 63) / 64);
        ia = t.ga1 - t.ga0;
        ib = t.gb1 - t.gb0;
        flops += 2.0 * (double)t.M * (double)t.N * (double)t.K;
      }
    }
    int total_flag, total_tiles, total_ia, total_ib;
    const int pos = block_scan(flag, ired, &total_flag);
    const int tpos = block_scan(tiles, ired, &total_tiles);
    const int apos = block_scan(ia, ired, &total_ia);
    const int bpos = block_scan(ib, ired, &total_ib);
    if (flag) {
      flagged[nflag + pos] = s;
      tile_end[nflag + pos] = ntile + tpos + tiles;
      item_end_a[nflag + pos] = nia + apos + ia;
      item_end_b[nflag + pos] = nib + bpos + ib;
    }
    nflag += total_flag;
    ntile += total_tiles;
    nia += total_ia;
    nib += total_ib;
  }
  norm = block_sum(norm, dred);
  err_split = block_sum(err_split, dred);
  err_after = block_sum(err_after, dred);
  flops = block_sum(flops, dred);
  {
    // maximum of the per-sector estimates
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
    __syncthreads();
    if ((tid & 31) == 0) dred[tid >> 5] = worst;
    __syncthreads();
    for (int w = 0; w < kThreads / 32; w++) worst = fmax(worst, dred[w]);
  }
  if (tid == 0) {
    auto rel = [&](double e2) { return e2 > 0.0 ? (norm > 0.0 ? sqrt(e2 / norm) : INFINITY) : 0.0; };
    rec->err_est = rel(err_after);
    rec->split_err_est = rel(err_split);
    rec->max_sector_est = worst;
    rec->fallback_flops = flops;
    rec->rtol = rtol;
    rec->nsectors = nsec;
    rec->nfallback = nflag;
    rec->within = rec->err_est <= rtol;
    rec->slices = slices;
    __threadfence();
    rec->valid = 1;
    if (!(rec->err_est <= rtol)) atomicCAS(status + 1, 0, 1);
  }
}

}  // namespace

cudaError_t launch_split_check(const SplitSector *sectors, int64_t nsec, const int32_t *ea, const int32_t *eb,
                               const int32_t *emax, const float *normsq, double *secv, int32_t *flagged,
                               int32_t *tile_end, int32_t *item_end_a, int32_t *item_end_b, SplitRecord *rec,
                               double eta_split, double eta_fp64, double rtol, int slices, int *status,
                               cudaStream_t stream) {
  if (nsec <= 0) return cudaSuccess;
  if (nsec > INT32_MAX) return cudaErrorInvalidValue;
  split_check_kernel<<<(unsigned)nsec, kThreads, 0, stream>>>(sectors, (int)nsec, ea, eb, emax, normsq, secv, flagged,
                                                              tile_end, item_end_a, item_end_b, rec, eta_split,
                                                              eta_fp64, rtol, slices, status);
  return cudaGetLastError();
}

}  // namespace ytn
