// Split-precision grouped GEMM over the charge sectors of a contraction on the
// 5th-generation tensor cores (tcgen05, accumulators in tensor memory, operands
// fed by bulk TMA copies), with FP64 results.
//
// Operands are the BF16 slices written by split_kernels.cu: A_q ~ 2^(e_i - 8)
// sum_p A_p and B_q ~ 2^(f_j - 8) sum_q B_q, with slice p (0-based) an integer
// digit times 2^{-8p}. C_q = 2^(e_i + f_j - 16) sum_{p + q <= s - 1} A_p B_q^T,
// where s is the number of slices used (products of order p + q >= s are
// dropped, as in the Ozaki scheme).
//
// Accumulation, per 128 x 128 output tile:
//   E2 = A_0 B_0                     order 0, exact in FP32 per K chunk of 64
//   E3 = A_0 B_1 + A_1 B_0           order 1, exact (an integer times 2^-8)
//   E4 = A_0 B_2 + A_1 B_1 + A_2 B_0 order 2, exact (an integer times 2^-16)
//   R  = every kept product of order >= 3, FP32 over the whole tile
// Chunk sums stay below 2^24 units of their lowest bit (3 * 64 * 255^2 < 2^24), so
// the three exact accumulators are exact; after each chunk the epilogue warps
// read them from tensor memory and add them into a 64-bit fixed-point accumulator
// (units of 2^-24 of the order-0 product). R, at most 2^-24 of the result, is
// rounded in FP32 and read once per tile. The result is converted to FP64 and
// scaled by 2^(e_i + f_j - 40). Tensor memory: E2 [0,128), E3 [128,256),
// E4 [256,384), R [384,512).
//
// Roles (one CTA per SM, persistent over the host-ordered tile list):
//   warp 0     bulk-copy producer: per K stage of 32, one copy of the A block and
//              one of the B block (s slices each, 8 KB per slice) into a
//              double-buffered shared-memory ring;
//   warp 1     MMA issuer (one thread): tcgen05.mma kind::f16, M = N = 128, K = 16;
//              inside a chunk the R products are issued first, so that the drain
//              of the previous chunk's exact accumulators overlaps tensor work;
//   warps 2-3  idle;
//   warps 4-15 epilogue: chunk drains and the FP64 output (three warps per
//              32-lane quarter of tensor memory, 40, 40 and 48 columns), which
//              keeps the 64-bit accumulators in registers under the 128-register
//              budget of a 512-thread CTA.
// Every wait is bounded; on expiry the kernel records a status code, stops
// issuing work, waits (bounded) for its own copies and MMAs and frees tensor
// memory before returning.
#include <cuda_runtime.h>

#include "kernels.hpp"

namespace ytn {

namespace {

constexpr int kThreads = 512;     // 16 warps
constexpr int kFirstEpiWarp = 4;  // warps 4..15: epilogue
constexpr int kEpiWarps = 12;
constexpr int kStagesRing = 2;
constexpr int kSlotBytes = 2 * kBlockBytes;
constexpr int kChunk = 2;         // K stages per exact-accumulation chunk (K 64)
constexpr uint32_t kColE2 = 0, kColE3 = 128, kColE4 = 256, kColR = 384;
constexpr uint32_t kMaxPolls = 1u << 26;
constexpr int kSmemBytes = kStagesRing * kSlotBytes + 1024 + 256;

// instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, N = 128, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

enum Bar { kFull0 = 0, kEmpty0 = 2, kEFull = 4, kEEmpty = 5, kRFull = 6, kREmpty = 7, kDone = 8, kNumBars = 9 };

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Bounded wait for the phase of parity `parity` to complete. Returns false (and
// records `code` in the status word and the CTA's abort flag) when the bound is
// reached or another role has aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag, int *status,
                                          int code) {
  for (uint32_t i = 0; i < kMaxPolls; i++) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((i & 63) == 63 && *abort_flag) return false;
  }
  *abort_flag = 1;
  atomicCAS(status, 0, code);
  return false;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// Shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row groups 512 B apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) | ((uint64_t)1 << 46) |
         ((uint64_t)4 << 61);
}

__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&r)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__global__ void __launch_bounds__(kThreads, 1)
    gemm_split_kernel(const SplitSector *__restrict__ sectors, const SplitTile *__restrict__ tiles, int ntiles,
                      const uint8_t *__restrict__ sa, const uint8_t *__restrict__ sb, const int32_t *__restrict__ ea,
                      const int32_t *__restrict__ eb, double *__restrict__ wc, int s, int *status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kStagesRing * kSlotBytes);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 16);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto bar = [&](int i) { return smem_u32(&bars[i]); };

  if (threadIdx.x == 0) {
    for (int i = 0; i < kStagesRing; i++) {
      mbar_init(bar(kFull0 + i), 1);
      mbar_init(bar(kEmpty0 + i), 1);
    }
    mbar_init(bar(kEFull), 1);
    mbar_init(bar(kEEmpty), kEpiWarps);
    mbar_init(bar(kRFull), 1);
    mbar_init(bar(kREmpty), kEpiWarps);
    mbar_init(bar(kDone), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      const uint32_t bytes = (uint32_t)s * kSliceBytes;
      uint32_t g = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const SplitTile tl = tiles[t];
        const SplitSector sc = sectors[tl.sector];
        const uint8_t *ablk = sa + sc.sa_off + (int64_t)tl.mt * sc.ks * kBlockBytes;
        const uint8_t *bblk = sb + sc.sb_off + (int64_t)tl.nt * sc.ks * kBlockBytes;
        for (int kt = 0; kt < sc.ks && ok; kt++, g++) {
          const int slot = g & 1;
          ok = mbar_wait(bar(kEmpty0 + slot), ((g >> 1) & 1) ^ 1, abort_flag, status, 1);
          if (!ok) break;
          uint8_t *dst = smem + slot * kSlotBytes;
          mbar_expect_tx(bar(kFull0 + slot), 2 * bytes);
          bulk_g2s(smem_u32(dst), ablk + (int64_t)kt * kBlockBytes, bytes, bar(kFull0 + slot));
          bulk_g2s(smem_u32(dst + kBlockBytes), bblk + (int64_t)kt * kBlockBytes, bytes, bar(kFull0 + slot));
        }
      }
      // no copy may still be in flight when the CTA exits
      for (uint32_t k = 1; k <= 2 && k <= g; k++) {
        const uint32_t gg = g - k;
        mbar_wait(bar(kFull0 + (gg & 1)), (gg >> 1) & 1, abort_flag, status, 2);
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      uint32_t g = 0, cc = 0, tcount = 0;
      bool ok = true;
      const uint32_t slot_base = smem_u32(smem);
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, tcount++) {
        const SplitSector sc = sectors[tiles[t].sector];
        const int nchunks = (sc.ks + kChunk - 1) / kChunk;
        for (int c = 0; c < nchunks && ok; c++, cc++) {
          const int st0 = c * kChunk, st1 = min(sc.ks, st0 + kChunk);
          for (int st = st0; st < st1; st++, g++) {
            const int slot = g & 1;
            ok = mbar_wait(bar(kFull0 + slot), (g >> 1) & 1, abort_flag, status, 3);
            if (!ok) break;
            tc_fence_after();
            const uint32_t aS = slot_base + slot * kSlotBytes, bS = aS + kBlockBytes;
            const bool first = st == st0, last = st == st1 - 1;
            auto mma = [&](uint32_t col, int p, int q, int ks, uint32_t acc) {
              umma(tmem + col, sdesc(aS + p * kSliceBytes + ks * 32), sdesc(bS + q * kSliceBytes + ks * 32), acc);
            };
            // orders 0, 1, 2 into the exact accumulators; `fresh` starts a new chunk
            auto issue_E = [&](bool fresh) {
              for (int ks = 0; ks < 2; ks++) {
                const uint32_t acc = (fresh && ks == 0) ? 0u : 1u;
                mma(kColE2, 0, 0, ks, acc);
                mma(kColE3, 0, 1, ks, acc);
                mma(kColE3, 1, 0, ks, 1u);
                mma(kColE4, 0, 2, ks, acc);
                mma(kColE4, 1, 1, ks, 1u);
                mma(kColE4, 2, 0, ks, 1u);
              }
            };
            // orders 3 .. s-1 into R; `fresh` starts a new tile
            auto issue_R = [&](bool fresh) {
              for (int ks = 0; ks < 2; ks++)
                for (int L = 3; L <= s - 1; L++)
                  for (int p = (L > s - 1 ? L - (s - 1) : 0); p <= L && p <= s - 1; p++)
                    mma(kColR, p, L - p, ks, (fresh && ks == 0 && L == 3 && p == 0) ? 0u : 1u);
            };
            auto wait_e_empty = [&]() {
              if (cc >= 1) {
                ok = mbar_wait(bar(kEEmpty), (cc - 1) & 1, abort_flag, status, 5);
                tc_fence_after();
              }
            };
            if (first && c == 0) {
              // new tile: exact accumulators after the previous chunk's drain, R after
              // the previous tile's R was read
              wait_e_empty();
              if (!ok) break;
              issue_E(true);
              if (tcount >= 1) {
                ok = mbar_wait(bar(kREmpty), (tcount - 1) & 1, abort_flag, status, 4);
                if (!ok) break;
                tc_fence_after();
              }
              issue_R(true);
              if (last) umma_commit(bar(kEFull));
            } else if (first) {
              issue_R(false);
              wait_e_empty();
              if (!ok) break;
              issue_E(true);
              if (last) umma_commit(bar(kEFull));
            } else {
              issue_E(false);
              umma_commit(bar(kEFull));
              issue_R(false);
            }
            umma_commit(bar(kEmpty0 + slot));
            if (last && c == nchunks - 1) umma_commit(bar(kRFull));
          }
        }
      }
      // every issued MMA has completed before tensor memory is released
      umma_commit(bar(kDone));
      mbar_wait(bar(kDone), 0, abort_flag, status, 6);
    }
  } else if (warp >= kFirstEpiWarp) {
    // ---------------------------------------------------------------- epilogue
    // three warps per 32-lane quarter of tensor memory; columns [40 t, 40 t + w)
    // with w = 40, 40, 48 for t = 0, 1, 2
    const int quarter = warp & 3, third = (warp - kFirstEpiWarp) >> 2;
    const int rl = quarter * 32 + lane;          // row inside the tile (tensor memory lane)
    const int c0 = third * 40;                   // first column of this thread
    const int ngroups = third == 2 ? 12 : 10;    // groups of 4 columns
    const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);
    uint32_t cc = 0, tcount = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, tcount++) {
      const SplitTile tl = tiles[t];
      const SplitSector sc = sectors[tl.sector];
      const int nchunks = (sc.ks + kChunk - 1) / kChunk;
      long long acc[48];
#pragma unroll
      for (int j = 0; j < 48; j++) acc[j] = 0;
      for (int c = 0; c < nchunks && ok; c++, cc++) {
        ok = mbar_wait(bar(kEFull), cc & 1, abort_flag, status, 7);
        if (!ok) break;
        tc_fence_after();
#pragma unroll
        for (int g = 0; g < 12; g++) {
          if (g < ngroups) {
            uint32_t v2[4], v3[4], v4[4];
            tmem_ld4(lane_addr + kColE2 + c0 + g * 4, v2);
            tmem_ld4(lane_addr + kColE3 + c0 + g * 4, v3);
            tmem_ld4(lane_addr + kColE4 + c0 + g * 4, v4);
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 4; i++) {
              const long long x2 = __float2int_rn(__uint_as_float(v2[i]));
              const long long x3 = __float2int_rn(__uint_as_float(v3[i]) * 256.0f);
              const long long x4 = __float2int_rn(__uint_as_float(v4[i]) * 65536.0f);
              acc[g * 4 + i] += (x2 << 24) + (x3 << 16) + (x4 << 8);
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(kEEmpty));
      }
      if (!ok) break;
      ok = mbar_wait(bar(kRFull), tcount & 1, abort_flag, status, 8);
      if (!ok) break;
      tc_fence_after();
#pragma unroll
      for (int g = 0; g < 6; g++) {
        if (g < ngroups / 2) {
          uint32_t vr[8];
          tmem_ld8(lane_addr + kColR + c0 + g * 8, vr);
          tmem_wait_ld();
#pragma unroll
          for (int i = 0; i < 8; i++) acc[g * 8 + i] += __float2ll_rn(__uint_as_float(vr[i]) * 16777216.0f);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(kREmpty));
      // C = acc * 2^(e_i + f_j - 40)
      const int row = tl.mt * kSplitBM + rl;
      if (row < sc.M) {
        const int ei = ea[sc.ea_off + row];
        double *crow = wc + sc.c_off + (int64_t)row * sc.N;
        const int n0 = tl.nt * kSplitBM + c0;
        const int32_t *fcol = eb + sc.eb_off + n0;
#pragma unroll
        for (int j = 0; j < 48; j++) {
          if (j < ngroups * 4 && n0 + j < sc.N) {
            // acc * 2^e as two exact power-of-two factors (covers |e| <= 2044)
            const int e = min(max(ei + __ldg(fcol + j) - 40, -2044), 2046);
            const int e1 = e >> 1, e2 = e - e1;
            crow[n0 + j] = __ll2double_rn(acc[j]) * __longlong_as_double((long long)(e1 + 1023) << 52) *
                           __longlong_as_double((long long)(e2 + 1023) << 52);
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 2) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

}  // namespace

cudaError_t launch_gemm_split(const SplitSector *sectors, const SplitTile *tiles, int64_t ntiles, const uint8_t *sa,
                              const uint8_t *sb, const int32_t *ea, const int32_t *eb, double *wc, int slices,
                              int *status, int num_sms, cudaStream_t stream) {
  if (ntiles <= 0) return cudaSuccess;
  if (ntiles > INT32_MAX || slices < 4 || slices > kSlices) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(gemm_split_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  if (e != cudaSuccess) return e;
  const int grid = (int)std::min<int64_t>(ntiles, num_sms);
  gemm_split_kernel<<<grid, kThreads, kSmemBytes, stream>>>(sectors, tiles, (int)ntiles, sa, sb, ea, eb, wc, slices,
                                                            status);
  return cudaGetLastError();
}

}  // namespace ytn
