// Data movers of the contraction path and of fuse / unfuse (Sec. II.B: the
// "permutes, reshapes, and copies" that fill the fused storage), plus the trace.
//
// One launch runs every piece of a phase. A CTA takes one work item: up to 32
// pieces (see CopyJob) with at most 4096 elements in all, staged whole in
// shared memory. The dense side of each piece (a contiguous range of its
// block) is moved linearly; the strided side is visited in its own order, so
// that consecutive threads touch consecutive addresses along its innermost
// dim. Index arithmetic per element is one multiply-high division per dim; the
// reads are asynchronous copies into shared memory, a whole item in flight.
// HBM-bound: every element is read once and written once.
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.hpp"

namespace ytn {

namespace {

constexpr int kThreads = 256;
constexpr int kJobWords = (int)(sizeof(CopyJob) / 4);

__device__ __forceinline__ void cp_async8(double *smem_dst, const double *gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
               "l"(gsrc)
               : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Negation by the sign bit (an integer operation: this GPU's FP64 pipe is far
// slower than its memory system); exact, and it keeps NaN payloads.
constexpr unsigned long long kSignBit = 0x8000000000000000ull;

__device__ __forceinline__ double flip(double x, unsigned long long mask) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)mask);
}

// The parameters of one piece, in registers: the last ND of its dim slots.
template <int ND>
struct Piece {
  int64_t g_off, d_off;
  int p;       // the piece's start in the staging buffer
  int negmode; // 0: as is; 1: negated (fermionic swap gate); 2: odd source offsets
               // negated (imaginary parts of interleaved complex data: conj)
  int ext[ND], gstr[ND], lstr[ND], shf[ND];
  uint32_t mag[ND];

  __device__ __forceinline__ void load(const CopyJob &J) {
    g_off = J.g_off;
    d_off = J.d_off;
    p = J.p;
    negmode = J.negate;
#pragma unroll
    for (int i = 0; i < ND; i++) {
      const int k = kMaxCopyDims - ND + i;
      ext[i] = J.ext[k];
      gstr[i] = J.gstr[k];
      lstr[i] = J.lstr[k];
      mag[i] = J.mag[k];
      shf[i] = J.shf[k];
    }
  }

  // Element l of the piece (in strided-side order): its offsets on the strided
  // side (global, from g_off) and on the dense side (from the piece's start).
  __device__ __forceinline__ void offsets(uint32_t l, int64_t &go, int &lo) const {
    go = 0;
    lo = 0;
#pragma unroll
    for (int i = ND - 1; i > 0; i--) {
      const uint32_t q = (l + __umulhi(l, mag[i])) >> shf[i];
      const int r = (int)(l - q * (uint32_t)ext[i]);
      go += (int64_t)r * gstr[i];
      lo += r * lstr[i];
      l = q;
    }
    go += (int64_t)l * gstr[0];
    lo += (int)l * lstr[0];
  }
};

// Calls body(P, l, e) for every element e of the item's flat range
// [w0, w1) of this warp: lanes take consecutive elements of one piece at a time
// (l: the element's index in its piece), so that a warp's accesses to the
// strided side follow that side's innermost dim. A piece's parameters are read
// from shared memory once per warp and piece.
template <int ND, class Body>
__device__ __forceinline__ void for_warp_range(const CopyJob *Js, int nj, int w0, int w1, Body body) {
  if (w0 >= w1) return;
  const int lane = threadIdx.x & 31;
  // first piece: the last one starting at or before w0
  int j = 31 - __clz(__ballot_sync(0xffffffffu, lane < nj && Js[lane].p <= w0));
  for (int e0 = w0; e0 < w1; j++) {
    Piece<ND> P;
    P.load(Js[j]);
    const int seg_end = min(w1, P.p + Js[j].size);
#pragma unroll 4
    for (int e = e0 + lane; e < seg_end; e += 32) body(P, e - P.p, e);
    e0 = seg_end;
  }
}

// DENSE_SRC (mode 2): read linearly, write in destination order; else
// (mode 3) read in source order, write linearly. The reads are asynchronous
// copies straight into shared memory, all of an item's in flight at once.
// Each warp takes one eighth of the item's elements in both phases.
template <int ND, bool DENSE_SRC>
__device__ __forceinline__ void stage_item(const CopyJob *Js, int nj, int total, const double *__restrict__ src,
                                           double *__restrict__ dst, double *stage) {
  constexpr int kWarps = kThreads / 32;
  const int per_warp = (total + kWarps - 1) / kWarps;
  const int w0 = min(total, (int)(threadIdx.x >> 5) * per_warp), w1 = min(total, w0 + per_warp);
  if (DENSE_SRC) {
    for_warp_range<ND>(Js, nj, w0, w1, [&](const Piece<ND> &P, int l, int e) {
      cp_async8(stage + e, src + P.d_off + l);
    });
  } else {
    for_warp_range<ND>(Js, nj, w0, w1, [&](const Piece<ND> &P, int l, int e) {
      int64_t go;
      int lo;
      P.offsets((uint32_t)l, go, lo);
      const int at = P.p + lo;
      if ((unsigned)at < (unsigned)total) cp_async8(stage + at, src + P.g_off + go);
    });
  }
  cp_async_wait_all();
  __syncthreads();
  if (DENSE_SRC) {
    for_warp_range<ND>(Js, nj, w0, w1, [&](const Piece<ND> &P, int l, int e) {
      int64_t go;
      int lo;
      P.offsets((uint32_t)l, go, lo);
      const int at = P.p + lo;
      const bool neg = P.negmode == 1 || (P.negmode == 2 && ((P.d_off + lo) & 1));
      if ((unsigned)at < (unsigned)total) dst[P.g_off + go] = flip(stage[at], neg ? kSignBit : 0ull);
    });
  } else {
    for_warp_range<ND>(Js, nj, w0, w1, [&](const Piece<ND> &P, int l, int e) {
      dst[P.d_off + l] = flip(stage[e], P.negmode == 1 ? kSignBit : 0ull);
    });
  }
}

template <int ND>
__device__ __forceinline__ void stage_dispatch(bool dense_src, const CopyJob *Js, int nj, int total,
                                               const double *src, double *dst, double *stage) {
  if (dense_src) stage_item<ND, true>(Js, nj, total, src, dst, stage);
  else stage_item<ND, false>(Js, nj, total, src, dst, stage);
}

// One work item: its pieces' parameters into shared memory, then the staged move.
// MAXND: the most dims an item of the launch has (the host reads it from the job
// table). Instantiated for at most 4 dims the kernel needs 48 registers instead
// of 64 and fits five CTAs per SM instead of four.
template <int MAXND>
__device__ __forceinline__ void run_item(const CopyJob *__restrict__ jobs, const CopyItem &it,
                                         const double *__restrict__ src, double *__restrict__ dst, CopyJob *Js,
                                         double *stage) {
  const int nj = it.njobs, total = it.total, nd = it.kind & 255, mode = it.kind >> 8;
  // the planner never makes other items, and the host never launches an item with
  // more dims than MAXND
  if (nj < 1 || nj > kStageJobs || total < 1 || total > kStageElems || nd < 1 || nd > MAXND) return;
  {
    const int32_t *s = reinterpret_cast<const int32_t *>(jobs + it.job);
    int32_t *d = reinterpret_cast<int32_t *>(Js);
    for (int w = threadIdx.x; w < nj * kJobWords; w += kThreads) d[w] = s[w];
  }
  __syncthreads();
  const bool dense_src = mode == 2;
  switch (nd) {
    case 1: stage_dispatch<1>(dense_src, Js, nj, total, src, dst, stage); break;
    case 2: stage_dispatch<2>(dense_src, Js, nj, total, src, dst, stage); break;
    case 3: stage_dispatch<3>(dense_src, Js, nj, total, src, dst, stage); break;
    case 4: stage_dispatch<4>(dense_src, Js, nj, total, src, dst, stage); break;
    default:
      if constexpr (MAXND > 4) {
        switch (nd) {
          case 5: stage_dispatch<5>(dense_src, Js, nj, total, src, dst, stage); break;
          case 6: stage_dispatch<6>(dense_src, Js, nj, total, src, dst, stage); break;
          case 7: stage_dispatch<7>(dense_src, Js, nj, total, src, dst, stage); break;
          default: stage_dispatch<8>(dense_src, Js, nj, total, src, dst, stage); break;
        }
      }
      break;
  }
}

template <int MAXND>
__global__ void __launch_bounds__(kThreads, MAXND <= 4 ? 5 : 4) copy_kernel(const CopyJob *__restrict__ jobs,
                                                                           const CopyItem *__restrict__ items,
                                                                           const double *__restrict__ src,
                                                                           double *__restrict__ dst) {
  __shared__ CopyJob Js[kStageJobs];
  __shared__ double stage[kStageElems];
  run_item<MAXND>(jobs, items[blockIdx.x], src, dst, Js, stage);
}

// Gathers of the sectors that the split path's accuracy check flagged (FP64
// fallback): a persistent grid walks the flagged sectors' work items (each
// sector's items are [first[q], first[q] + count), the running counts over the
// flagged sectors in item_end). With no flagged sector every CTA returns at once.
__global__ void __launch_bounds__(kThreads, 4) copy_flagged_kernel(const CopyJob *__restrict__ jobs,
                                                                   const CopyItem *__restrict__ items,
                                                                   const SplitSector *__restrict__ sectors, int which,
                                                                   const int32_t *__restrict__ flagged,
                                                                   const int32_t *__restrict__ item_end,
                                                                   const SplitRecord *__restrict__ rec,
                                                                   const double *__restrict__ src,
                                                                   double *__restrict__ dst) {
  __shared__ CopyJob Js[kStageJobs];
  __shared__ double stage[kStageElems];
  const int nflag = rec->nfallback;
  if (nflag <= 0) return;
  const int total = item_end[nflag - 1];
  for (int t = blockIdx.x; t < total; t += gridDim.x) {
    int lo = 0, hi = nflag - 1;   // first flagged sector whose items end after t
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (item_end[mid] > t) hi = mid;
      else lo = mid + 1;
    }
    const SplitSector &sc = sectors[flagged[lo]];
    const int first = which == 0 ? sc.ga0 : sc.gb0;
    const int local = t - (lo > 0 ? item_end[lo - 1] : 0);
    __syncthreads();   // the previous item's shared memory is no longer read
    run_item<kMaxCopyDims>(jobs, items[first + local], src, dst, Js, stage);
  }
}

// Zero fill of the flagged sectors' FP64 sector matrices (partially populated
// operands) before their gathers.
__global__ void __launch_bounds__(kThreads) zero_flagged_kernel(const SectorDev *__restrict__ sectors,
                                                                const int32_t *__restrict__ flagged,
                                                                const SplitRecord *__restrict__ rec, double *wa,
                                                                double *wb, int zero_a, int zero_b) {
  const int nflag = rec->nfallback;
  for (int k = blockIdx.x; k < nflag; k += gridDim.x) {
    const SectorDev s = sectors[flagged[k]];
    const int64_t na = zero_a ? (int64_t)s.M * s.K : 0, nb = zero_b ? (int64_t)s.K * s.N : 0;
    for (int64_t e = threadIdx.x; e < na; e += kThreads) wa[s.a_off + e] = 0.0;
    for (int64_t e = threadIdx.x; e < nb; e += kThreads) wb[s.b_off + e] = 0.0;
  }
}

// Trace: thread per output element; contributing blocks and diagonal elements
// are summed in a fixed order.
__global__ void __launch_bounds__(128) trace_kernel(const TraceOut *__restrict__ outs,
                                                    const TraceContrib *__restrict__ contribs,
                                                    const double *__restrict__ src,
                                                    double *__restrict__ dst) {
  const TraceOut o = outs[blockIdx.x];
  for (int e = threadIdx.x; e < o.nrest; e += blockDim.x) {
    int idx[kMaxCopyDims];
    int r = e;
    for (int i = o.nrd - 1; i >= 0; i--) {
      idx[i] = r % o.rext[i];
      r /= o.rext[i];
    }
    double sum = 0.0;
    for (int c = o.first; c < o.first + o.ncontrib; c++) {
      const TraceContrib &tc = contribs[c];
      int64_t base = tc.src_off;
      for (int i = 0; i < o.nrd; i++) base += (int64_t)idx[i] * tc.rstr[i];
      int P = 1;
      for (int k = 0; k < tc.ndiag; k++) P *= tc.dext[k];
      for (int d = 0; d < P; d++) {
        int rem = d;
        int64_t off = base;
        for (int k = tc.ndiag - 1; k >= 0; k--) {
          const int dk = rem % tc.dext[k];
          rem /= tc.dext[k];
          off += (int64_t)dk * tc.dstr[k];
        }
        sum += src[off];
      }
    }
    dst[o.dst_off + e] = sum;
  }
}

// Scatter-combine of a complex product: the doubled real C_q holds the four
// real products in quadrants; one CTA per C block writes re = P00 - P11 and
// im = P01 + P10 (absent quadrants, from a real operand, count as zero) as
// interleaved complex elements. Reads follow the block's innermost dim along a
// row of C_q; the writes are consecutive 16-byte pairs.
__global__ void __launch_bounds__(256) cscatter_kernel(const CScatterJob *__restrict__ jobs,
                                                       const double *__restrict__ P, double *__restrict__ C) {
  const CScatterJob J = jobs[blockIdx.x];
  double2 *out = reinterpret_cast<double2 *>(C) + J.dst;
  for (int e = threadIdx.x; e < J.n; e += blockDim.x) {
    int r = e;
    int64_t so = J.src;
    for (int i = J.nd - 1; i >= 0; i--) {
      const int x = r % J.ext[i];
      r /= J.ext[i];
      so += (int64_t)x * J.sstr[i];
    }
    double re = P[so], im = 0.0;
    if (J.q11 >= 0) re -= P[so + J.q11];
    if (J.q01 >= 0) im += P[so + J.q01];
    if (J.q10 >= 0) im += P[so + J.q10];
    out[e] = make_double2(re, im);
  }
}

}  // namespace

cudaError_t launch_cscatter(const CScatterJob *jobs, int64_t njobs, const double *wc, double *c,
                            cudaStream_t stream) {
  if (njobs <= 0) return cudaSuccess;
  if (njobs > INT32_MAX) return cudaErrorInvalidValue;
  cscatter_kernel<<<(unsigned)njobs, 256, 0, stream>>>(jobs, wc, c);
  return cudaGetLastError();
}

cudaError_t launch_copy(const CopyJob *jobs, const CopyItem *items, int64_t nitems, const double *src,
                        double *dst, cudaStream_t stream, int max_nd) {
  if (nitems <= 0) return cudaSuccess;
  if (nitems > INT32_MAX || max_nd < 1 || max_nd > kMaxCopyDims) return cudaErrorInvalidValue;
  if (max_nd <= 4) copy_kernel<4><<<(unsigned)nitems, kThreads, 0, stream>>>(jobs, items, src, dst);
  else copy_kernel<kMaxCopyDims><<<(unsigned)nitems, kThreads, 0, stream>>>(jobs, items, src, dst);
  return cudaGetLastError();
}

cudaError_t launch_trace(const TraceOut *outs, int64_t nout, const TraceContrib *contribs,
                         const double *src, double *dst, cudaStream_t stream) {
  if (nout <= 0) return cudaSuccess;
  if (nout > INT32_MAX) return cudaErrorInvalidValue;
  trace_kernel<<<(unsigned)nout, 128, 0, stream>>>(outs, contribs, src, dst);
  return cudaGetLastError();
}

cudaError_t launch_gather_flagged(const CopyJob *jobs, const CopyItem *items_a, const CopyItem *items_b,
                                  const SplitSector *sp_sectors, const SectorDev *sectors, const int32_t *flagged,
                                  const int32_t *item_end_a, const int32_t *item_end_b, const SplitRecord *rec,
                                  const double *a, const double *b, double *wa, double *wb, bool zero_a, bool zero_b,
                                  int num_sms, cudaStream_t stream) {
  const unsigned grid = (unsigned)std::max(1, num_sms) * 4;
  if (zero_a || zero_b) zero_flagged_kernel<<<grid, kThreads, 0, stream>>>(sectors, flagged, rec, wa, wb, zero_a, zero_b);
  copy_flagged_kernel<<<grid, kThreads, 0, stream>>>(jobs, items_a, sp_sectors, 0, flagged, item_end_a, rec, a, wa);
  copy_flagged_kernel<<<grid, kThreads, 0, stream>>>(jobs, items_b, sp_sectors, 1, flagged, item_end_b, rec, b, wb);
  return cudaGetLastError();
}

}  // namespace ytn
