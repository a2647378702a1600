// Fused split of the split-precision path: BF16 slices built straight from the
// tensors' blocks, with no FP64 sector matrix in between (Sec. II.B: the blocks
// are fused into one matrix per charge sector; here the fused matrix only ever
// exists as its slices).
//
// A work item is 32 rows of one operand (a quarter of a 128-row slice tile) and
// 128 of K (four K stages). Its segments (planner: SliceSeg) are the parts of the
// blocks that fall inside it. Both kernels load the whole item into a shared-memory
// tile of raw FP64 bits with asynchronous copies, every element in flight at once:
//   split_rowmax_kernel: the item's row maxima of the biased exponent, combined
//                        over the row's items into its scale exponent with
//                        atomicMax (and into the operand's largest);
//   split_digits_kernel: the balanced digits at that scale, written as s BF16
//                        slices in the tensor cores' swizzled layout.
// HBM traffic per operand element: 8 bytes read twice and 2 s bytes written (the
// staged path moves 8 bytes in and out of an FP64 sector matrix first, then reads
// it twice).
//
// Every warp copies an equal share of the item: its segments are cut along the
// direction the walk steps in. The walk follows the block's contiguous direction:
// when its innermost free stride is the smaller the lanes are rows and the warp
// steps along K, else the lanes are K and the warp steps along the rows. A lane's
// offset is decomposed once (mixed radix over the block's free or contracted dims)
// and the stepped one is carried from index to index, so that an element costs one
// asynchronous copy and an add.
#include <cuda_runtime.h>

#include <climits>

#include "kernels.hpp"
#include "split_digits.cuh"

namespace ytn {

namespace {

constexpr int kThreads = 256;
constexpr int kPitch = kItemK + 1; // tile row pitch in elements (odd: fewer bank conflicts)

__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
               "l"(gsrc)
               : "memory");
}

struct Smem {
  unsigned long long tile[kItemRows][kPitch];
  int red[kThreads / 32][kItemRows];
  int rexp[kItemRows];
};

// A mixed-radix index over up to kFusedDims dims (row-major, outer first) and its
// element offset inside the block, stepped by one with carries (no division). The
// dims sit in the last slots (unused outer slots: extent 1, stride 0), so that every
// index below is a constant and the walker lives in registers. Offsets inside a
// block fit 32 bits, one step past its last element included (the planner keeps
// blocks spanning more than 2^30 elements off the fused path).
struct Walker {
  int32_t ext[kFusedDims], idx[kFusedDims], st[kFusedDims];
  int32_t off;

  __device__ __forceinline__ void start(int i, int nd, const int32_t *e, const int64_t *s) {
    off = 0;
#pragma unroll
    for (int d = kFusedDims - 1; d >= 0; d--) {
      const int k = d - (kFusedDims - nd);   // the dim in this slot, if any
      ext[d] = k >= 0 ? e[k] : 1;
      st[d] = k >= 0 ? (int32_t)s[k] : 0;
      const int q = i / ext[d];
      idx[d] = i - q * ext[d];
      off += idx[d] * st[d];
      i = q;
    }
  }
  // the next index (carries past the last valid index are harmless: the offset is
  // not used any more)
  __device__ __forceinline__ void step() {
    idx[kFusedDims - 1]++;
    off += st[kFusedDims - 1];
#pragma unroll
    for (int t = kFusedDims - 1; t > 0; t--) {
      if (idx[t] == ext[t]) {
        idx[t] = 0;
        off -= ext[t] * st[t];
        idx[t - 1]++;
        off += st[t - 1];
      }
    }
  }
};

// Units [u0, u1) of a segment into the tile. rfast: a unit is one column of K, the
// lanes its rows; else a unit is one row, the lanes its K (four per lane).
__device__ __forceinline__ void load_units(Smem &sm, const SliceSeg &g, int u0, int u1, int lane,
                                           const double *__restrict__ X) {
  const int r0 = g.r0, nr = g.r1 - g.r0, k0 = g.k0, kc = g.k1 - g.k0;
  const double *base = X + g.boff;
  if (g.rfast) {
    Walker kw;
    kw.start(g.kbase + u0, g.nk, g.kext, g.kst);
    const double *rb = base;
    if (lane < nr) {
      Walker rw;
      rw.start(g.ibase + lane, g.nf, g.fext, g.fst);
      rb += rw.off;
    }
    for (int k = u0; k < u1; k++) {
      if (lane < nr) cp_async8(&sm.tile[r0 + lane][k0 + k], rb + kw.off);
      kw.step();
    }
  } else {
    int32_t ko[kItemK / 32];
#pragma unroll
    for (int q = 0; q < kItemK / 32; q++) {
      ko[q] = 0;
      if (lane + 32 * q < kc) {
        Walker kw;
        kw.start(g.kbase + lane + 32 * q, g.nk, g.kext, g.kst);
        ko[q] = kw.off;
      }
    }
    Walker rw;
    rw.start(g.ibase + u0, g.nf, g.fext, g.fst);
    for (int r = u0; r < u1; r++) {
#pragma unroll
      for (int q = 0; q < kItemK / 32; q++)
        if (lane + 32 * q < kc) cp_async8(&sm.tile[r0 + r][k0 + lane + 32 * q], base + rw.off + ko[q]);
      rw.step();
    }
  }
}

// The item's 32 x 128 elements into the tile (zero where no block lies). Each warp
// takes an equal share [lo, hi) of the item's cost (warp-wide copy steps, summed
// over the segments in order): the units of a segment whose starting cost falls in
// that share. A unit u of a segment with starting cost c0 and unit cost w starts at
// c0 + u w, so the warp's units are those with ceil((lo - c0) / w) <= u <
// ceil((hi - c0) / w), and every unit goes to exactly one warp. Each lane looks at
// one segment of a group of 32 and the warp takes the ones that meet its share in
// order; offsets are decomposed once per lane and part, and stepped after that.
__device__ __forceinline__ void load_item(Smem &sm, const SliceItem &it, const SliceSeg *__restrict__ segs,
                                          const double *__restrict__ X) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int kWarps = kThreads / 32;
  if (!it.full) {
    for (int w = tid; w < kItemRows * kItemK; w += kThreads) sm.tile[w / kItemK][w % kItemK] = 0ull;
    __syncthreads();   // zero fill before the copies land
  }
  const int lo = (warp * it.cost) / kWarps, hi = ((warp + 1) * it.cost) / kWarps;
  const SliceSeg *sg = segs + it.seg0;
  for (int j0 = 0; j0 < it.nseg && hi > lo; j0 += 32) {
    const int j = j0 + lane;
    int c0 = INT_MAX, c1 = INT_MAX;
    if (j < it.nseg) {
      c0 = sg[j].cost0;
      c1 = j + 1 < it.nseg ? sg[j + 1].cost0 : it.cost;
    }
    uint32_t meet = __ballot_sync(0xffffffffu, c0 < hi && c1 > lo);
    const bool past = __any_sync(0xffffffffu, j < it.nseg && c1 >= hi);
    while (meet) {
      const int b = __ffs(meet) - 1;
      meet &= meet - 1;
      const int s0 = __shfl_sync(0xffffffffu, c0, b);
      const SliceSeg &g = sg[j0 + b];
      const int nr = g.r1 - g.r0, kc = g.k1 - g.k0;
      const int w = g.rfast ? 1 : (kc + 31) / 32;
      const int nu = g.rfast ? kc : nr;
      const int u0 = lo > s0 ? (lo - s0 + w - 1) / w : 0;
      const int u1 = min(nu, (hi - s0 + w - 1) / w);
      if (u0 < u1) load_units(sm, g, u0, u1, lane, X);
    }
    if (past) break;   // later segments start at or beyond hi
  }
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads) split_rowmax_kernel(const SplitOperand *__restrict__ ops,
                                                                const SliceItem *__restrict__ items,
                                                                const SliceSeg *__restrict__ segs,
                                                                const double *__restrict__ a,
                                                                const double *__restrict__ b,
                                                                int32_t *__restrict__ ea, int32_t *__restrict__ eb,
                                                                int32_t *__restrict__ emax) {
  __shared__ Smem sm;
  const SliceItem it = items[blockIdx.x];
  const SplitOperand o = ops[it.op];
  const bool isA = (it.op & 1) == 0;
  load_item(sm, it, segs, isA ? a : b);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // lanes are rows (bank-friendly), warps take 16 elements each of the row; K
  // stages past the operand's last are not in the tile (a multiple of 32 of K)
  const int kcv = min(kItemK, o.ks * kSplitBK - it.kq * kItemK);
  int m = 0;
  if (warp * (kItemK / 8) < kcv)
#pragma unroll
    for (int j = 0; j < kItemK / 8; j++)
      m = max(m, biased_exp(__longlong_as_double((long long)sm.tile[lane][warp * (kItemK / 8) + j])));
  sm.red[warp][lane] = m;
  __syncthreads();
  if (warp == 0) {
    int r = sm.red[0][lane];
#pragma unroll
    for (int w = 1; w < kThreads / 32; w++) r = max(r, sm.red[w][lane]);
    const int row = it.rt * kSplitBM + it.quarter * kItemRows + lane;
    int mine = INT_MIN;
    if (row < o.rows) {
      atomicMax((isA ? ea : eb) + o.exp_off + row, r - 1021);
      mine = r - 1021;
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) mine = max(mine, __shfl_xor_sync(0xffffffffu, mine, s));
    if (lane == 0 && mine != INT_MIN) atomicMax(emax + it.op, mine);
  }
}

__global__ void __launch_bounds__(kThreads) split_digits_kernel(const SplitOperand *__restrict__ ops,
                                                                const SliceItem *__restrict__ items,
                                                                const SliceSeg *__restrict__ segs,
                                                                const double *__restrict__ a,
                                                                const double *__restrict__ b,
                                                                const int32_t *__restrict__ ea,
                                                                const int32_t *__restrict__ eb,
                                                                uint8_t *__restrict__ sa, uint8_t *__restrict__ sb,
                                                                int s) {
  __shared__ Smem sm;
  const SliceItem it = items[blockIdx.x];
  const SplitOperand o = ops[it.op];
  const bool isA = (it.op & 1) == 0;
  const int tid = threadIdx.x;
  const int row0 = it.rt * kSplitBM + it.quarter * kItemRows;
  if (tid < kItemRows) sm.rexp[tid] = row0 + tid < o.rows ? ((isA ? ea : eb) + o.exp_off)[row0 + tid] : -1021;
  load_item(sm, it, segs, isA ? a : b);
  uint8_t *S = (isA ? sa : sb) + o.slice_off;
  // tasks: (stage, row, 16-byte chunk), a warp covering 8 rows of one stage (512
  // contiguous bytes of each slice)
  for (int task = tid; task < kItemRows * (kItemK / 8); task += kThreads) {
    const int stage = task >> 7, rr = (task >> 2) & (kItemRows - 1), c = task & 3;
    const int kt = it.kq * (kItemK / kSplitBK) + stage;
    if (kt >= o.ks) continue;   // K stages past the operand do not exist
    uint32_t packed[kSlices][4];
    slice_digits8(&sm.tile[rr][stage * kSplitBK + c * 8], sm.rexp[rr], s, packed);
    uint8_t *blk = S + ((int64_t)it.rt * o.ks + kt) * kBlockBytes;
    store_slices(blk, slice_pos(it.quarter * kItemRows + rr, c), s, packed);
  }
}

}  // namespace

cudaError_t launch_split_blocks(const SplitOperand *ops, const SliceItem *items, int64_t nitems,
                                const SliceSeg *segs, const double *a, const double *b, int32_t *ea, int32_t *eb,
                                int32_t *emax, uint8_t *sa, uint8_t *sb, int slices, cudaStream_t stream) {
  if (nitems <= 0) return cudaSuccess;
  if (nitems > INT32_MAX || slices < 1 || slices > kSlices) return cudaErrorInvalidValue;
  split_rowmax_kernel<<<(unsigned)nitems, kThreads, 0, stream>>>(ops, items, segs, a, b, ea, eb, emax);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  split_digits_kernel<<<(unsigned)nitems, kThreads, 0, stream>>>(ops, items, segs, a, b, ea, eb, sa, sb, slices);
  return cudaGetLastError();
}

}  // namespace ytn
