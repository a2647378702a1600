// Grouped FP64 GEMM over the charge sectors of a contraction (Sec. II.B: the
// fused matrices are multiplied sector by sector, C_q = A_q B_q), on the FP64
// tensor cores (DMMA, mma.sync m8n8k4 f64).
//
// One launch covers every sector: the grid is the host-built tile list
// (sector, m-tile, n-tile), largest K first so that long tiles start early.
// Each CTA computes one tile of C_q over the full K (no split-K), so every
// output element has one fixed summation order: results do not depend on the
// schedule or on what else runs on the GPU. The tile edge (64, or 32 for small
// and thin sectors) is chosen per sector by the planner from the sector's M and
// N, so that many small sectors do not pay for 64x64 tiles.
//
// On GB300 the FP64 rate (DMMA and DFMA alike, about 1 TFLOP/s for the whole
// GPU) is low enough that this kernel is bound by the FP64 pipe even at 64x64
// tiles; operands are staged through padded shared memory with a register
// prefetch of the next K step.
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.hpp"

namespace ytn {

namespace {

constexpr int BK = 16, PAD = 4;
constexpr int kThreads = 128;

__device__ __forceinline__ void dmma(double (&c)[2], double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(c[0]), "+d"(c[1])
               : "d"(a), "d"(b));
}

// Load one BK-slice of the A (or B) tile into registers: T x 16 elements, T/8 per
// thread. kmajor: element (r, k) at base[r * ld + k]; else at base[k * ld + r].
template <int T>
__device__ __forceinline__ void load_tile(double (&v)[T / 8], const double *__restrict__ base, int ld, bool kmajor,
                                          int rows, int r0, int k0, int K) {
  const int t = threadIdx.x;
  if (kmajor) {
    const int k = t & 15;
#pragma unroll
    for (int i = 0; i < T / 8; i++) {
      const int r = (t >> 4) + 8 * i;
      const int gr = r0 + r, gk = k0 + k;
      v[i] = (gr < rows && gk < K) ? __ldg(base + (int64_t)gr * ld + gk) : 0.0;
    }
  } else {
    const int r = t & (T - 1);
#pragma unroll
    for (int i = 0; i < T / 8; i++) {
      const int k = t / T + (kThreads / T) * i;
      const int gr = r0 + r, gk = k0 + k;
      v[i] = (gr < rows && gk < K) ? __ldg(base + (int64_t)gk * ld + gr) : 0.0;
    }
  }
}

template <int T>
__device__ __forceinline__ void store_tile(double (*s)[64 + PAD], const double (&v)[T / 8], bool kmajor) {
  const int t = threadIdx.x;
  if (kmajor) {
    const int k = t & 15;
#pragma unroll
    for (int i = 0; i < T / 8; i++) s[k][(t >> 4) + 8 * i] = v[i];
  } else {
    const int r = t & (T - 1);
#pragma unroll
    for (int i = 0; i < T / 8; i++) s[t / T + (kThreads / T) * i][r] = v[i];
  }
}

// One T x T tile of C_q (T = 64 or 32): four warps of (T/2) x (T/2), each a grid of
// (T/16) x (T/16) DMMA 8x8 blocks.
template <int T>
__device__ __forceinline__ void gemm_tile(const SectorDev &s, const GemmTile &tl, const double *__restrict__ wa,
                                          const double *__restrict__ wb, double *__restrict__ wc,
                                          double (*As)[BK][64 + PAD], double (*Bs)[BK][64 + PAD]) {
  constexpr int NB = T / 16;
  const int M = s.M, N = s.N, K = s.K;
  const int m0 = tl.mt * T, n0 = tl.nt * T;
  const double *A = wa + s.a_off;
  const double *B = wb + s.b_off;
  const int lda = s.a_kmajor ? K : M;
  const int ldb = s.b_kmajor ? K : N;
  const bool akm = s.a_kmajor != 0, bkm = s.b_kmajor != 0;

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wm = (warp >> 1) * (T / 2), wn = (warp & 1) * (T / 2);
  double acc[NB][NB][2];
#pragma unroll
  for (int i = 0; i < NB; i++)
#pragma unroll
    for (int j = 0; j < NB; j++) acc[i][j][0] = acc[i][j][1] = 0.0;

  double ra[T / 8], rb[T / 8];
  const int nk = (K + BK - 1) / BK;
  if (nk > 0) {
    load_tile<T>(ra, A, lda, akm, M, m0, 0, K);
    load_tile<T>(rb, B, ldb, bkm, N, n0, 0, K);
    store_tile<T>(As[0], ra, akm);
    store_tile<T>(Bs[0], rb, bkm);
  }
  __syncthreads();
  for (int kt = 0; kt < nk; kt++) {
    const int cur = kt & 1;
    const bool more = kt + 1 < nk;
    if (more) {
      load_tile<T>(ra, A, lda, akm, M, m0, (kt + 1) * BK, K);
      load_tile<T>(rb, B, ldb, bkm, N, n0, (kt + 1) * BK, K);
    }
#pragma unroll
    for (int kk = 0; kk < BK; kk += 4) {
      double af[NB], bf[NB];
#pragma unroll
      for (int i = 0; i < NB; i++) af[i] = As[cur][kk + (lane & 3)][wm + i * 8 + (lane >> 2)];
#pragma unroll
      for (int j = 0; j < NB; j++) bf[j] = Bs[cur][kk + (lane & 3)][wn + j * 8 + (lane >> 2)];
#pragma unroll
      for (int i = 0; i < NB; i++)
#pragma unroll
        for (int j = 0; j < NB; j++) dmma(acc[i][j], af[i], bf[j]);
    }
    if (more) {
      store_tile<T>(As[cur ^ 1], ra, akm);
      store_tile<T>(Bs[cur ^ 1], rb, bkm);
    }
    __syncthreads();
  }
  double *C = wc + s.c_off;
#pragma unroll
  for (int i = 0; i < NB; i++) {
    const int m = m0 + wm + i * 8 + (lane >> 2);
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < NB; j++) {
      const int n = n0 + wn + j * 8 + 2 * (lane & 3);
      if (n < N) C[(int64_t)m * N + n] = acc[i][j][0];
      if (n + 1 < N) C[(int64_t)m * N + n + 1] = acc[i][j][1];
    }
  }
}

__global__ void __launch_bounds__(kThreads) gemm_fp64_kernel(const SectorDev *__restrict__ sectors,
                                                             const GemmTile *__restrict__ tiles,
                                                             const double *__restrict__ wa,
                                                             const double *__restrict__ wb,
                                                             double *__restrict__ wc) {
  __shared__ double As[2][BK][64 + PAD];
  __shared__ double Bs[2][BK][64 + PAD];
  const GemmTile tl = tiles[blockIdx.x];
  const SectorDev s = sectors[tl.sector];
  if (tl.size == 32) gemm_tile<32>(s, tl, wa, wb, wc, As, Bs);
  else gemm_tile<64>(s, tl, wa, wb, wc, As, Bs);
}

// FP64 recomputation of the sectors that the split path's accuracy check
// flagged: a persistent grid walks the flagged sectors' 64 x 64 tiles, whose list
// the check wrote on the device (tile_end: running tile counts per flagged
// sector). With no flagged sector every CTA returns at once.
__global__ void __launch_bounds__(kThreads) gemm_fp64_redo_kernel(const SectorDev *__restrict__ sectors,
                                                                  const int32_t *__restrict__ flagged,
                                                                  const int32_t *__restrict__ tile_end,
                                                                  const SplitRecord *__restrict__ rec,
                                                                  const double *__restrict__ wa,
                                                                  const double *__restrict__ wb,
                                                                  double *__restrict__ wc) {
  __shared__ double As[2][BK][64 + PAD];
  __shared__ double Bs[2][BK][64 + PAD];
  const int nflag = rec->nfallback;
  if (nflag <= 0) return;
  const int total = tile_end[nflag - 1];
  for (int t = blockIdx.x; t < total; t += gridDim.x) {
    int lo = 0, hi = nflag - 1;   // first flagged sector whose tiles end after t
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (tile_end[mid] > t) hi = mid;
      else lo = mid + 1;
    }
    const int local = t - (lo > 0 ? tile_end[lo - 1] : 0);
    const SectorDev s = sectors[flagged[lo]];
    const int nt = (s.N + 63) / 64;
    const GemmTile tl{flagged[lo], local / nt, local % nt, 64};
    gemm_tile<64>(s, tl, wa, wb, wc, As, Bs);
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_gemm_fp64_redo(const SectorDev *sectors, const int32_t *flagged, const int32_t *tile_end,
                                  const SplitRecord *rec, const double *wa, const double *wb, double *wc,
                                  int num_sms, cudaStream_t stream) {
  gemm_fp64_redo_kernel<<<(unsigned)std::max(1, num_sms) * 4, kThreads, 0, stream>>>(sectors, flagged, tile_end, rec,
                                                                                    wa, wb, wc);
  return cudaGetLastError();
}

cudaError_t launch_gemm_fp64(const SectorDev *sectors, const GemmTile *tiles, int64_t ntiles,
                             const double *wa, const double *wb, double *wc, cudaStream_t stream) {
  if (ntiles <= 0) return cudaSuccess;
  if (ntiles > INT32_MAX) return cudaErrorInvalidValue;
  gemm_fp64_kernel<<<(unsigned)ntiles, kThreads, 0, stream>>>(sectors, tiles, wa, wb, wc);
  return cudaGetLastError();
}

}  // namespace ytn
