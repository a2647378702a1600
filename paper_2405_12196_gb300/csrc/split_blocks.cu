// Fused split of the split-precision path: BF16 slices built straight from the
// tensors' blocks, with no FP64 sector matrix in between (Sec. II.B: the blocks
// are fused into one matrix per charge sector; here the fused matrix only ever
// exists as its slices).
//
// A work item is 32 rows of one operand (a quarter of a 128-row slice tile) and
// 128 of K (four K stages). Its segments (planner: SliceSeg) are the parts of the
// blocks that fall inside it.
//   split_rowmax_kernel: the item's row maxima of the biased exponent, read
//                        straight into registers (two items per CTA), combined
//                        over the row's items into its scale exponent with
//                        atomicMax (and into the operand's largest);
//   split_digits_kernel: the whole item loaded into a shared-memory tile of raw
//                        FP64 bits with asynchronous copies, every element in
//                        flight at once, then the balanced digits at the row
//                        scales, written as s BF16 slices in the tensor cores'
//                        swizzled layout.
// Both take the items of a range [items, items + nitems): the whole list, or one
// sector group of the pipelined variant (its instances launched beside the split
// GEMM are sized to share an SM with a GEMM CTA).
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
// load (or asynchronous copy) and an add.
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

// The digits kernel's shared memory: the item's tile of raw FP64 bits and its
// rows' scale exponents (33.2 KB).
struct __align__(16) Smem {
  unsigned long long tile[kItemRows][kPitch];
  int rexp[kItemRows];
};

// Offset of index i over the nd dims of one side of a block (extents e and strides
// s, outer first; nd <= kFusedDims): nd - 1 divisions. Offsets inside a block fit
// 32 bits, one step past its last element included (the planner keeps blocks
// spanning more than 2^30 elements off the fused path).
__device__ __forceinline__ int32_t side_offset(int i, int nd, const int32_t *e, const int64_t *s) {
  int32_t off = 0;
#pragma unroll
  for (int d = kFusedDims - 1; d >= 1; d--)
    if (d < nd) {
      const int q = i / e[d];
      off += (i - q * e[d]) * (int32_t)s[d];
      i = q;
    }
  return nd >= 1 ? off + i * (int32_t)s[0] : 0;
}

// A mixed-radix index over the ND dims of one side of a block (row-major, outer
// first) and its offset, stepped by one with carries (no division).
template <int ND>
struct Stepper {
  static constexpr int kN = ND > 0 ? ND : 1;
  int32_t ext[kN], idx[kN], st[kN];
  int32_t off;

  __device__ __forceinline__ void start(int i, const int32_t *e, const int64_t *s) {
    off = 0;
#pragma unroll
    for (int d = ND - 1; d >= 0; d--) {
      ext[d] = e[d];
      st[d] = (int32_t)s[d];
      if (d > 0) {
        const int q = i / ext[d];
        idx[d] = i - q * ext[d];
        i = q;
      } else {
        idx[d] = i;
      }
      off += idx[d] * st[d];
    }
  }
  // the next index (carries past the last valid index are harmless: the offset is
  // not used any more)
  __device__ __forceinline__ void step() {
    if (ND == 0) return;
    idx[ND - 1]++;
    off += st[ND - 1];
#pragma unroll
    for (int t = ND - 1; t > 0; t--) {
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
// lanes its rows; else a unit is one row, the lanes its K (four per lane). ND: the
// dims of the stepped side (K when rfast, else the rows).
template <int ND>
__device__ __forceinline__ void load_units(Smem &sm, const SliceSeg &g, int u0, int u1, int lane,
                                           const double *__restrict__ X) {
  const int r0 = g.r0, nr = g.r1 - g.r0, k0 = g.k0, kc = g.k1 - g.k0;
  const double *base = X + g.boff;
  if (g.rfast) {
    Stepper<ND> kw;
    kw.start(g.kbase + u0, g.kext, g.kst);
    const double *rb = base;
    if (lane < nr) rb += side_offset(g.ibase + lane, g.nf, g.fext, g.fst);
    unsigned long long *t = &sm.tile[r0 + lane][k0];
    for (int k = u0; k < u1; k++) {
      if (lane < nr) cp_async8(t + k, rb + kw.off);
      kw.step();
    }
  } else {
    int32_t ko[kItemK / 32];
#pragma unroll
    for (int q = 0; q < kItemK / 32; q++)
      ko[q] = lane + 32 * q < kc ? side_offset(g.kbase + lane + 32 * q, g.nk, g.kext, g.kst) : 0;
    Stepper<ND> rw;
    rw.start(g.ibase + u0, g.fext, g.fst);
    for (int r = u0; r < u1; r++) {
      const double *rb = base + rw.off;
      unsigned long long *t = &sm.tile[r0 + r][k0 + lane];
#pragma unroll
      for (int q = 0; q < kItemK / 32; q++)
        if (lane + 32 * q < kc) cp_async8(t + 32 * q, rb + ko[q]);
      rw.step();
    }
  }
}

__device__ __forceinline__ void load_units_any(Smem &sm, const SliceSeg &g, int u0, int u1, int lane,
                                               const double *__restrict__ X) {
  switch (g.rfast ? g.nk : g.nf) {
    case 0: load_units<0>(sm, g, u0, u1, lane, X); break;
    case 1: load_units<1>(sm, g, u0, u1, lane, X); break;
    case 2: load_units<2>(sm, g, u0, u1, lane, X); break;
    default: load_units<3>(sm, g, u0, u1, lane, X); break;
  }
}

// A warp's share of an item: f(g, u0, u1) for the units [u0, u1) of each segment g
// whose units start inside the cost range [lo, hi) (for_warp_share: an equal share
// of the item's cost, warp-wide copy steps summed over the segments in order, per
// warp). A unit u of a segment with starting cost c0
// and unit cost w starts at c0 + u w, so the warp's units are those with
// ceil((lo - c0) / w) <= u < ceil((hi - c0) / w), and every unit goes to exactly one
// warp. Each lane looks at one segment of a group of 32 and the warp takes the ones
// that meet its share in order.
template <class F>
__device__ __forceinline__ void for_cost_range(const SliceItem &it, const SliceSeg *__restrict__ segs, int lo, int hi,
                                               F f) {
  const int lane = threadIdx.x & 31;
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
      if (u0 < u1) f(g, u0, u1);
    }
    if (past) break;   // later segments start at or beyond hi
  }
}

template <class F>
__device__ __forceinline__ void for_warp_share(const SliceItem &it, const SliceSeg *__restrict__ segs, F f) {
  const int warp = threadIdx.x >> 5;
  constexpr int kWarps = kThreads / 32;
  for_cost_range(it, segs, (warp * it.cost) / kWarps, ((warp + 1) * it.cost) / kWarps, f);
}

// The item's 32 x 128 elements into the tile (zero where no block lies), offsets
// decomposed once per lane and part and stepped after that.
__device__ __forceinline__ void load_item(Smem &sm, const SliceItem &it, const SliceSeg *__restrict__ segs,
                                          const double *__restrict__ X) {
  const int tid = threadIdx.x, lane = tid & 31;
  if (!it.full) {   // the whole tile, pitch padding included, in 16-byte stores
    uint4 *z = reinterpret_cast<uint4 *>(&sm.tile[0][0]);
    for (int w = tid; w < (int)(sizeof(sm.tile) / 16); w += kThreads) z[w] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();   // zero fill before the copies land
  }
  for_warp_share(it, segs, [&](const SliceSeg &g, int u0, int u1) { load_units_any(sm, g, u0, u1, lane, X); });
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
  __syncthreads();
}

// The biased exponent of the double at p, from its upper word.
__device__ __forceinline__ int biased_exp_at(const double *p) {
  return (int)((__ldg(reinterpret_cast<const unsigned int *>(p) + 1) >> 20) & 0x7FF);
}

// Row maxima of the biased exponent over units [u0, u1) of a segment, combined into
// rmax (shared memory, one per row of the item). rfast: each lane keeps its row's
// maximum over the K columns it steps through, eight loads in flight; else each row
// is one step, its maximum reduced over the warp. ND: the dims of the stepped side.
template <int ND>
__device__ __forceinline__ void rowmax_units(int *rmax, const SliceSeg &g, int u0, int u1, int lane,
                                             const double *__restrict__ X) {
  const int r0 = g.r0, nr = g.r1 - g.r0, kc = g.k1 - g.k0;
  const double *base = X + g.boff;
  if (g.rfast) {
    const bool act = lane < nr;
    Stepper<ND> kw;
    kw.start(g.kbase + u0, g.kext, g.kst);
    const double *rb = base;
    if (act) rb += side_offset(g.ibase + lane, g.nf, g.fext, g.fst);
    int m = 0;
    int k = u0;
    for (; k + 8 <= u1; k += 8) {
      int x[8];
#pragma unroll
      for (int q = 0; q < 8; q++) {
        x[q] = act ? biased_exp_at(rb + kw.off) : 0;
        kw.step();
      }
#pragma unroll
      for (int q = 0; q < 8; q++) m = max(m, x[q]);
    }
    for (; k < u1; k++) {
      if (act) m = max(m, biased_exp_at(rb + kw.off));
      kw.step();
    }
    if (act) atomicMax(rmax + r0 + lane, m);
  } else {
    int32_t ko[kItemK / 32];
#pragma unroll
    for (int q = 0; q < kItemK / 32; q++)
      ko[q] = lane + 32 * q < kc ? side_offset(g.kbase + lane + 32 * q, g.nk, g.kext, g.kst) : 0;
    Stepper<ND> rw;
    rw.start(g.ibase + u0, g.fext, g.fst);
    for (int r = u0; r < u1; r++) {
      const double *rb = base + rw.off;
      int m = 0;
#pragma unroll
      for (int q = 0; q < kItemK / 32; q++)
        if (lane + 32 * q < kc) m = max(m, biased_exp_at(rb + ko[q]));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (lane == 0) atomicMax(rmax + r0 + r, m);
      rw.step();
    }
  }
}

// Row maxima of the biased exponent over each item's elements, combined over the
// row's items into its scale exponent (E = max - 1021, so that |x| < 2^(E - 1))
// with atomicMax, and into the operand's largest. Rows without elements in the item
// count as 0 (as zeros do). No staging: the elements are read straight into
// registers. A CTA takes two consecutive items (their records and segment tables
// read together), its warps equal shares of their summed cost; eight CTAs per SM (32
// registers) keep the most loads in flight (measured against six and four).
// BESIDE: the instance launched beside the split GEMM (pipelined variant), the same
// code with the SM's shared-memory carveout at its maximum (set at context
// creation), so that the SMs it runs on stay configured for the GEMM's CTAs.
constexpr int kRowmaxItems = 2;

template <bool BESIDE>
__global__ void __launch_bounds__(kThreads, 8) split_rowmax_kernel(const SplitOperand *__restrict__ ops,
                                                                   const SliceItem *__restrict__ items, int nitems,
                                                                   const SliceSeg *__restrict__ segs,
                                                                   const double *__restrict__ a,
                                                                   const double *__restrict__ b,
                                                                   int32_t *__restrict__ ea, int32_t *__restrict__ eb,
                                                                   int32_t *__restrict__ emax) {
  __shared__ int rmax[kRowmaxItems][kItemRows];
  __shared__ SliceItem rec[kRowmaxItems];
  const int i0 = blockIdx.x * kRowmaxItems, ni = min(kRowmaxItems, nitems - i0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid < kRowmaxItems * kItemRows) rmax[tid / kItemRows][tid % kItemRows] = 0;
  if (tid < ni * (int)(sizeof(SliceItem) / 4))
    reinterpret_cast<int32_t *>(rec)[tid] = reinterpret_cast<const int32_t *>(items + i0)[tid];
  __syncthreads();
  const SliceItem &it0 = rec[0], &it1 = rec[ni > 1 ? 1 : 0];
  const int c0 = it0.cost, total = c0 + (ni > 1 ? it1.cost : 0);
  constexpr int kWarps = kThreads / 32;
  const int lo = (warp * total) / kWarps, hi = ((warp + 1) * total) / kWarps;
#pragma unroll 1
  for (int t = 0; t < kRowmaxItems; t++) {
    if (t >= ni) break;
    const SliceItem &it = t == 0 ? it0 : it1;
    const int base = t == 0 ? 0 : c0;
    const int l = max(lo - base, 0), h = min(hi - base, it.cost);
    if (l >= h) continue;
    const double *X = (it.op & 1) == 0 ? a : b;
    int *rm = rmax[t];
    for_cost_range(it, segs, l, h, [&](const SliceSeg &g, int u0, int u1) {
      switch (g.rfast ? g.nk : g.nf) {
        case 0: rowmax_units<0>(rm, g, u0, u1, lane, X); break;
        case 1: rowmax_units<1>(rm, g, u0, u1, lane, X); break;
        case 2: rowmax_units<2>(rm, g, u0, u1, lane, X); break;
        default: rowmax_units<3>(rm, g, u0, u1, lane, X); break;
      }
    });
  }
  __syncthreads();
  if (warp < ni) {   // warp t flushes item t's rows
    const SliceItem &it = warp == 0 ? it0 : it1;
    const bool isA = (it.op & 1) == 0;
    const SplitOperand &o = ops[it.op];
    const int row = it.rt * kSplitBM + it.quarter * kItemRows + lane;
    int mine = INT_MIN;
    if (row < o.rows) {
      const int r = rmax[warp][lane];
      atomicMax((isA ? ea : eb) + o.exp_off + row, r - 1021);
      mine = r - 1021;
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) mine = max(mine, __shfl_xor_sync(0xffffffffu, mine, s));
    if (lane == 0 && mine != INT_MIN) atomicMax(emax + it.op, mine);
  }
}

// MINB: CTAs per SM the launch bounds ask for. 5: 48 registers (five CTAs per SM,
// as shared memory allows), the fastest alone; 6: 40
// registers, so that one CTA fits beside a split-GEMM CTA (576 threads x 96
// registers + 256 x 40 = 65,536; shared memory 198,912 + 34,176 bytes with the
// per-CTA reserve, within the SM's 233,472), for the slicing that runs beside the
// GEMM in the pipelined variant.
template <int MINB>
__global__ void __launch_bounds__(kThreads, MINB) split_digits_kernel(const SplitOperand *__restrict__ ops,
                                                                      const SliceItem *__restrict__ items,
                                                                      const SliceSeg *__restrict__ segs,
                                                                      const double *__restrict__ a,
                                                                      const double *__restrict__ b,
                                                                      const int32_t *__restrict__ ea,
                                                                      const int32_t *__restrict__ eb,
                                                                      uint8_t *__restrict__ sa,
                                                                      uint8_t *__restrict__ sb, int s) {
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

cudaError_t configure_split_blocks() {
  cudaError_t e = cudaFuncSetAttribute(split_rowmax_kernel<true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(split_digits_kernel<6>, cudaFuncAttributePreferredSharedMemoryCarveout,
                              cudaSharedmemCarveoutMaxShared);
}

cudaError_t launch_split_blocks(const SplitOperand *ops, const SliceItem *items, int64_t nitems,
                                const SliceSeg *segs, const double *a, const double *b, int32_t *ea, int32_t *eb,
                                int32_t *emax, uint8_t *sa, uint8_t *sb, int slices, bool beside_gemm,
                                cudaStream_t stream) {
  if (nitems <= 0) return cudaSuccess;
  if (nitems > INT32_MAX || slices < 1 || slices > kSlices) return cudaErrorInvalidValue;
  const unsigned g0 = (unsigned)((nitems + kRowmaxItems - 1) / kRowmaxItems);
  if (beside_gemm)
    split_rowmax_kernel<true><<<g0, kThreads, 0, stream>>>(ops, items, (int)nitems, segs, a, b, ea, eb, emax);
  else
    split_rowmax_kernel<false><<<g0, kThreads, 0, stream>>>(ops, items, (int)nitems, segs, a, b, ea, eb, emax);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (beside_gemm)
    split_digits_kernel<6><<<(unsigned)nitems, kThreads, 0, stream>>>(ops, items, segs, a, b, ea, eb, sa, sb, slices);
  else
    split_digits_kernel<5><<<(unsigned)nitems, kThreads, 0, stream>>>(ops, items, segs, a, b, ea, eb, sa, sb, slices);
  return cudaGetLastError();
}

}  // namespace ytn
