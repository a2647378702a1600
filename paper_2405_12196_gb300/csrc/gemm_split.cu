// Split-precision grouped GEMM over the charge sectors of a contraction on the
// 5th-generation tensor cores (tcgen05, accumulators in tensor memory, operands
// fed by bulk TMA copies), with FP64 results.
//
// Operands are the BF16 slices written by split_kernels.cu: A_q = 2^(e_i - 8)
// sum_p A_p and B_q = 2^(f_j - 8) sum_q B_q (up to the rounding of the last digit),
// with slice p a signed digit of magnitude <= 2^7 times 2^{-8p}.
// C_q = 2^(e_i + f_j - 16) sum_{p + q <= s - 1} A_p B_q^T, where s is the number of
// slices used (products of order p + q >= s are dropped, as in the Ozaki scheme).
//
// Accumulation, per 128 x 128 output tile:
//   E2 = A_0 B_0                     order 0, exact in FP32 per K chunk of 256
//   E3 = A_0 B_1 + A_1 B_0           order 1, exact (an integer times 2^-8)
//   E4 = A_0 B_2 + A_1 B_1 + A_2 B_0 order 2, exact (an integer times 2^-16)
//   R  = every kept product of order >= 3, FP32 per K chunk of 256
// A digit product is at most 2^14 in magnitude, so over a chunk of 256 the three
// exact accumulators stay within 3 * 256 * 2^14 < 2^24 units of their lowest bit
// and FP32 holds them exactly; after each chunk the epilogue warps read all four
// from tensor memory and add them into a 64-bit fixed-point accumulator (units
// of 2^-24 of the order-0 product). Only R, about 2^-24 of the result per K, is
// rounded in FP32, and only over 256 of K at a time (the tensor cores' FP32
// accumulation of mixed-magnitude products is not round-to-nearest, so its error
// grows with the number of additions). The result is converted to FP64 and
// scaled by 2^(e_i + f_j - 40). Tensor memory: E2 [0,128), E3 [128,256),
// E4 [256,384), R [384,512).
//
// Roles (one CTA per SM, persistent over the host-ordered tile list):
//   warp 0     bulk-copy producer: per K stage of 32, one copy of the A block and
//              one of the B block (s slices each, 8 KB per slice) into a
//              double-buffered shared-memory ring;
//   warp 1     MMA issuer (one thread): tcgen05.mma kind::f16, M = N = 128, K = 16;
//              the drain of the exact accumulators overlaps a chunk's last R
//              products, the drain of R the next chunk's first exact products;
//   warps 2-17 epilogue: chunk drains and the FP64 output (four warps per
//              32-lane quarter of tensor memory, 32 columns each; warp 2 also
//              allocates and frees tensor memory), which keeps the 64-bit
//              accumulators in registers under the 96-register budget of a
//              576-thread CTA. At five slices the drain of the exact accumulators
//              is not hidden behind the last stage's R products; four warps per
//              quarter instead of three shorten it.
// Every wait is bounded; on expiry the kernel records a status code, stops
// issuing work, waits (bounded) for its own copies and MMAs and frees tensor
// memory before returning.
#include <cuda_runtime.h>

#include "kernels.hpp"

namespace ytn {

namespace {

constexpr int kThreads = 576;     // 18 warps
constexpr int kFirstEpiWarp = 2;  // warps 2..17: epilogue
constexpr int kEpiWarps = 16;
constexpr int kStagesRing = 2;
constexpr int kSlotBytes = 2 * kBlockBytes;
constexpr int kChunk = 8;         // K stages per exact-accumulation chunk (K 256)
constexpr uint32_t kColE2 = 0, kColE3 = 128, kColE4 = 256, kColR = 384;
constexpr uint32_t kMaxPolls = 1u << 26;
constexpr int kSmemBytes = kStagesRing * kSlotBytes + 1024 + 256;

// instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M = 128; the
// N field (bits 17..22, N / 8) is set per tile: 128, or 64 for the narrow tiles
constexpr uint32_t kIdescBase = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 4) << 24);
__device__ __forceinline__ uint32_t idesc_for(int bn) { return kIdescBase | ((uint32_t)(bn >> 3) << 17); }

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

__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
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

// acc * 2^e as an FP64 value, rounded to nearest even. The bit pattern is built
// with integer operations (FP64 arithmetic is slow on this GPU); results outside
// the normal range take the FP64 path.
__device__ __forceinline__ double scaled_double(long long acc, int e) {
  if (acc == 0) return 0.0;
  const unsigned long long sign = acc < 0 ? (1ull << 63) : 0ull;
  const unsigned long long m = acc < 0 ? (unsigned long long)(-acc) : (unsigned long long)acc;
  const int lz = __clzll((long long)m);
  const unsigned long long mn = m << lz;           // leading one at bit 63
  unsigned long long mant = mn >> 11;               // 53 bits with the leading one
  const unsigned long long rem = mn & 0x7FFull;
  int be = 63 - lz + e + 1023;                      // biased exponent of the result
  if (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) {
    mant += 1ull;
    if (mant == (1ull << 53)) {
      mant >>= 1;
      be += 1;
    }
  }
  if (be >= 1 && be <= 2046)
    return __longlong_as_double((long long)(sign | ((unsigned long long)be << 52) | (mant & 0xFFFFFFFFFFFFFull)));
  const int ec = min(max(e, -2044), 2046), e1 = ec >> 1, e2 = ec - e1;
  return __ll2double_rn(acc) * __longlong_as_double((long long)(e1 + 1023) << 52) *
         __longlong_as_double((long long)(e2 + 1023) << 52);
}

// Descriptor offsets in the 16-byte units of the start-address field: one slice
// of A (8 KB) and one K step of 16 (32 bytes); B's slices lie 8 KB apart in a
// 128-wide tile and 4 KB apart in a 64-wide one (bsu). The shared-memory footprint
// stays below 256 KB, so additions never carry out of the 14-bit field.
constexpr uint64_t kSliceU = kSliceBytes >> 4, kStepU = 2;

// Orders 0, 1, 2 of one 32-wide K stage into the exact accumulators; `fresh`
// starts a new chunk. a0 / b0: descriptors of slice 0 of the stage.
__device__ __forceinline__ void issue_exact(uint32_t tmem, uint64_t a0, uint64_t b0, bool fresh, uint32_t idesc,
                                            uint64_t bsu) {
#pragma unroll
  for (int ks = 0; ks < 2; ks++) {
    const uint64_t a = a0 + ks * kStepU, b = b0 + ks * kStepU;
    const uint32_t acc = (fresh && ks == 0) ? 0u : 1u;
    umma(tmem + kColE2, a, b, idesc, acc);
    umma(tmem + kColE3, a, b + bsu, idesc, acc);
    umma(tmem + kColE3, a + kSliceU, b, idesc, 1u);
    umma(tmem + kColE4, a, b + 2 * bsu, idesc, acc);
    umma(tmem + kColE4, a + kSliceU, b + bsu, idesc, 1u);
    umma(tmem + kColE4, a + 2 * kSliceU, b, idesc, 1u);
  }
}

// Orders 3 .. S-1 of one stage into R; `fresh` starts a new chunk.
template <int S>
__device__ __forceinline__ void issue_rest(uint32_t tmem, uint64_t a0, uint64_t b0, bool fresh, uint32_t idesc,
                                           uint64_t bsu) {
#pragma unroll
  for (int ks = 0; ks < 2; ks++) {
    const uint64_t a = a0 + ks * kStepU, b = b0 + ks * kStepU;
#pragma unroll
    for (int L = 3; L <= S - 1; L++) {
#pragma unroll
      for (int p = 0; p <= L; p++) {
        if (p > S - 1 || L - p > S - 1) continue;
        const uint32_t acc = (fresh && ks == 0 && L == 3 && p == 0) ? 0u : 1u;
        umma(tmem + kColR, a + p * kSliceU, b + (L - p) * bsu, idesc, acc);
      }
    }
  }
}

// 2^k as an FP32 value for k <= 0 (0 below the normal range).
__device__ __forceinline__ float pow2f(int k) { return k >= -126 ? __int_as_float((k + 127) << 23) : 0.0f; }

// MIX: the tile list may hold 64-wide tiles (tile width read per tile); without it
// every tile is 128 wide and the widths are constants.
template <int S, bool MIX>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_split_kernel(const SplitSector *__restrict__ sectors, const SplitTile *__restrict__ tiles, int ntiles,
                      const uint8_t *__restrict__ sa, const uint8_t *__restrict__ sb, const int32_t *__restrict__ ea,
                      const int32_t *__restrict__ eb, const int32_t *__restrict__ emax, float *__restrict__ normsq,
                      double *__restrict__ wc, int *status) {
  constexpr int s = S;
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
        // a 64-wide tile reads one half (64 rows, 4 KB per slice) of a 128-row B block
        const bool narrow = MIX && tl.bn == 64;
        const uint8_t *bblk = sb + sc.sb_off + (int64_t)(narrow ? tl.nt >> 1 : tl.nt) * sc.ks * kBlockBytes +
                              (narrow ? (tl.nt & 1) * (kSliceBytes / 2) : 0);
        for (int kt = 0; kt < sc.ks && ok; kt++, g++) {
          const int slot = g & 1;
          ok = mbar_wait(bar(kEmpty0 + slot), ((g >> 1) & 1) ^ 1, abort_flag, status, 1);
          if (!ok) break;
          uint8_t *dst = smem + slot * kSlotBytes;
          mbar_expect_tx(bar(kFull0 + slot), narrow ? bytes + bytes / 2 : 2 * bytes);
          bulk_g2s(smem_u32(dst), ablk + (int64_t)kt * kBlockBytes, bytes, bar(kFull0 + slot));
          if (!narrow) {
            bulk_g2s(smem_u32(dst + kBlockBytes), bblk + (int64_t)kt * kBlockBytes, bytes, bar(kFull0 + slot));
          } else {
            for (int p = 0; p < s; p++)
              bulk_g2s(smem_u32(dst + kBlockBytes + p * (kSliceBytes / 2)),
                       bblk + (int64_t)kt * kBlockBytes + p * kSliceBytes, kSliceBytes / 2, bar(kFull0 + slot));
          }
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
        const SplitTile tlm = tiles[t];
        const SplitSector sc = sectors[tlm.sector];
        const int nchunks = (sc.ks + kChunk - 1) / kChunk;
        const bool narrow = MIX && tlm.bn == 64;
        const uint32_t idesc = idesc_for(narrow ? 64 : 128);
        const uint64_t bsu = narrow ? kSliceU / 2 : kSliceU;
        for (int c = 0; c < nchunks && ok; c++, cc++) {
          const int st0 = c * kChunk, st1 = min(sc.ks, st0 + kChunk);
          for (int st = st0; st < st1; st++, g++) {
            const int slot = g & 1;
            ok = mbar_wait(bar(kFull0 + slot), (g >> 1) & 1, abort_flag, status, 3);
            if (!ok) break;
            tc_fence_after();
            const uint32_t aS = slot_base + slot * kSlotBytes, bS = aS + kBlockBytes;
            const bool first = st == st0, last = st == st1 - 1;
            const uint64_t a0 = sdesc(aS), b0 = sdesc(bS);
            auto wait_e_empty = [&]() {
              if (cc >= 1) {
                ok = mbar_wait(bar(kEEmpty), (cc - 1) & 1, abort_flag, status, 5);
                tc_fence_after();
              }
            };
            // Every chunk starts all four accumulators afresh: the exact ones once the
            // previous chunk's exact drain is done, R once its R drain is done. The
            // exact accumulators are complete after the last stage's exact products,
            // so their drain overlaps that stage's R products; the drain of R
            // overlaps the next chunk's first exact products.
            if (first) {
              wait_e_empty();
              if (!ok) break;
              issue_exact(tmem, a0, b0, true, idesc, bsu);
              if (last) umma_commit(bar(kEFull));
              if (cc >= 1) {
                ok = mbar_wait(bar(kREmpty), (cc - 1) & 1, abort_flag, status, 4);
                if (!ok) break;
                tc_fence_after();
              }
              issue_rest<S>(tmem, a0, b0, true, idesc, bsu);
            } else {
              issue_exact(tmem, a0, b0, false, idesc, bsu);
              if (last) umma_commit(bar(kEFull));
              issue_rest<S>(tmem, a0, b0, false, idesc, bsu);
            }
            umma_commit(bar(kEmpty0 + slot));
            if (last) umma_commit(bar(kRFull));
          }
        }
      }
      // every issued MMA has completed before tensor memory is released
      umma_commit(bar(kDone));
      mbar_wait(bar(kDone), 0, abort_flag, status, 6);
    }
  } else if (warp >= kFirstEpiWarp) {
    // ---------------------------------------------------------------- epilogue
    // four warps per 32-lane quarter of tensor memory; columns [c0, c0 + w) with
    // w = 32 in a 128-wide tile and 16 in a 64-wide one
    const int quarter = warp & 3, part = (warp - kFirstEpiWarp) >> 2;
    const int rl = quarter * 32 + lane;          // row inside the tile (tensor memory lane)
    const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);
    uint32_t cc = 0, tcount = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, tcount++) {
      const SplitTile tl = tiles[t];
      const SplitSector sc = sectors[tl.sector];
      const bool narrow = MIX && tl.bn == 64;
      const int c0 = narrow ? part * 16 : part * 32;   // first column
      const int ngroups = narrow ? 4 : 8;              // groups of 4 columns
      const int nchunks = (sc.ks + kChunk - 1) / kChunk;
      long long acc[32];
#pragma unroll
      for (int j = 0; j < 32; j++) acc[j] = 0;
      for (int c = 0; c < nchunks && ok; c++, cc++) {
        ok = mbar_wait(bar(kEFull), cc & 1, abort_flag, status, 7);
        if (!ok) break;
        tc_fence_after();
#pragma unroll
        for (int g = 0; g < 8; g++) {
          if (g < ngroups) {
            uint32_t v2[4], v3[4], v4[4];
            tmem_ld4(lane_addr + kColE2 + c0 + g * 4, v2);
            tmem_ld4(lane_addr + kColE3 + c0 + g * 4, v3);
            tmem_ld4(lane_addr + kColE4 + c0 + g * 4, v4);
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 4; i++) {
              // order 0: |E2| <= 256 * 2^14 = 2^22, read from the bit pattern of
              // E2 + 1.5 * 2^23 (exact on the closed range: the pattern is linear in
              // the integer up to and including 2^24)
              const int x2 = __float_as_int(__uint_as_float(v2[i]) + 12582912.0f) - 0x4B400000;
              // order 1: |E3 * 2^8| <= 2 * 256 * 2^14 = 2^23
              const int x3 = __float2int_rn(__uint_as_float(v3[i]) * 256.0f);
              // order 2: |E4 * 2^16| <= 3 * 256 * 2^14 < 2^24
              const int x4 = __float2int_rn(__uint_as_float(v4[i]) * 65536.0f);
              // |x2 * 2^8 + x3| <= 2^30 + 2^23 < 2^31
              acc[g * 4 + i] += (long long)(x2 * 256 + x3) * 65536 + (long long)x4 * 256;
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(kEEmpty));
        ok = mbar_wait(bar(kRFull), cc & 1, abort_flag, status, 8);
        if (!ok) break;
        tc_fence_after();
#pragma unroll
        for (int g = 0; g < 4; g++) {
          if (g < ngroups / 2) {
            uint32_t vr[8];
            tmem_ld8(lane_addr + kColR + c0 + g * 8, vr);
            tmem_wait_ld();
            // |R| over one chunk <= 256 (4 * 2^14 * 2^-24 + 5 * 2^14 * 2^-32 + 6 * 2^14 * 2^-40)
            // < 1.02, so R * 2^24 fits 32 bits
#pragma unroll
            for (int i = 0; i < 8; i++)
              acc[g * 8 + i] += (long long)__float2int_rn(__uint_as_float(vr[i]) * 16777216.0f);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(kREmpty));
      }
      if (!ok) break;
      // C = acc * 2^(e_i + f_j - 40); beside it, the tile's share of the sector's
      // ||C_q||^2 relative to 4^(emax_A + emax_B) for the accuracy check, in FP32
      // (acc * 2^-40 from its two 32-bit halves, squared, scaled by powers of two)
      const int row = tl.mt * kSplitBM + rl;
      float ss = 0.0f;
      if (row < sc.M) {
        const int ei = ea[sc.ea_off + row];
        const int fmax = __ldg(emax + 2 * tl.sector + 1);
        double *crow = wc + sc.c_off + (int64_t)row * sc.N;
        const int n0 = tl.nt * (narrow ? 64 : kSplitBM) + c0;
        const int32_t *fcol = eb + sc.eb_off + n0;
#pragma unroll
        for (int j = 0; j < 32; j++) {
          if (j < ngroups * 4 && n0 + j < sc.N) {
            const int fj = __ldg(fcol + j);
            crow[n0 + j] = scaled_double(acc[j], ei + fj - 40);
            const float v = fmaf((float)(int)(acc[j] >> 32), 0x1p-8f, (float)(uint32_t)acc[j] * 0x1p-40f) *
                            pow2f(fj - fmax);
            ss = fmaf(v, v, ss);
          }
        }
        ss *= pow2f(2 * (ei - __ldg(emax + 2 * tl.sector)));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
      if (lane == 0 && ss > 0.0f) atomicAdd(normsq + tl.sector, ss);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 2) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

}  // namespace

// Opt the kernels in to their shared-memory size; once per device (a context
// does it at creation), so that launches stay free of non-stream calls.
cudaError_t configure_split_gemm() {
  for (auto kernel : {gemm_split_kernel<4, false>, gemm_split_kernel<5, false>, gemm_split_kernel<6, false>,
                      gemm_split_kernel<4, true>, gemm_split_kernel<5, true>, gemm_split_kernel<6, true>}) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    // all of the SM's unified memory as shared memory, so that a slicing CTA of the
    // pipelined split fits beside this kernel's CTA (the L1 share it leaves unused
    // is not read by this kernel: operands arrive by bulk copies)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_gemm_split(const SplitSector *sectors, const SplitTile *tiles, int64_t ntiles, const uint8_t *sa,
                              const uint8_t *sb, const int32_t *ea, const int32_t *eb, const int32_t *emax,
                              float *normsq, double *wc, int slices, int *status, int num_sms, bool mixed_widths,
                              cudaStream_t stream) {
  if (ntiles <= 0) return cudaSuccess;
  if (ntiles > INT32_MAX || slices < 4 || slices > kSlices) return cudaErrorInvalidValue;
  auto kernel = mixed_widths ? (slices == 4   ? gemm_split_kernel<4, true>
                                : slices == 5 ? gemm_split_kernel<5, true>
                                              : gemm_split_kernel<6, true>)
                             : (slices == 4   ? gemm_split_kernel<4, false>
                                : slices == 5 ? gemm_split_kernel<5, false>
                                              : gemm_split_kernel<6, false>);
  const int grid = (int)std::min<int64_t>(ntiles, num_sms);
  kernel<<<grid, kThreads, kSmemBytes, stream>>>(sectors, tiles, (int)ntiles, sa, sb, ea, eb, emax, normsq, wc,
                                                 status);
  return cudaGetLastError();
}

}  // namespace ytn
