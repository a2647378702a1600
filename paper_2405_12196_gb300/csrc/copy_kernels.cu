// Data movers of the contraction path and of fuse / unfuse (Sec. II.B: the
// "permutes, reshapes, and copies" that fill the fused storage), plus the trace.
//
// One launch runs every job of a phase: each CTA takes one work item (a range
// of rows or tiles of one block). HBM-bound: every element is read once and
// written once.
//   rows mode: the destination-contiguous dimension is also the source's
//     innermost one; warps copy whole rows with coalesced loads and stores.
//     Rows shorter than 16 elements are packed several to a warp.
//   tile mode: the two layouts have different contiguous dimensions; a 32x32
//     tile is staged through shared memory so that both the global loads and
//     the global stores are coalesced.
//   staged modes: blocks of at most a few thousand elements, up to 32 of them
//     per CTA, pass whole through shared memory: the contiguous side is moved
//     linearly, the strided side in its own coalescing order, so that one CTA
//     moves about 32 KB whatever the block shapes.
#include <cuda_runtime.h>

#include "kernels.hpp"

namespace ytn {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

__device__ __forceinline__ void row_offsets(const CopyJob &J, uint32_t row, int64_t &so, int64_t &dof) {
  so = J.src_off;
  dof = J.dst_off;
  for (int i = J.nd - 2; i >= 0; i--) {
    const uint32_t e = (uint32_t)J.ext[i];
    const uint32_t idx = row % e;
    row /= e;
    so += (int64_t)idx * J.sst[i];
    dof += (int64_t)idx * J.dst[i];
  }
}

// Element l (in the order of the job's dims) of a staged job: its offsets
// along the two sides, relative to the job's origins.
__device__ __forceinline__ void staged_offsets(const CopyJob &J, uint32_t l, int64_t &so, int64_t &dof) {
  so = 0;
  dof = 0;
  for (int i = J.nd - 1; i > 0; i--) {
    const uint32_t e = (uint32_t)J.ext[i];
    const uint32_t idx = l % e;
    l /= e;
    so += (int64_t)idx * J.sst[i];
    dof += (int64_t)idx * J.dst[i];
  }
  so += (int64_t)l * J.sst[0];
  dof += (int64_t)l * J.dst[0];
}

union CopySmem {
  double tile[kTile][kTile + 1];
  double stage[kStageElems];
};

__device__ __forceinline__ void copy_staged(const CopyJob *__restrict__ jobs, const CopyItem &it,
                                            const double *__restrict__ src, double *__restrict__ dst,
                                            CopyJob *Js, double *stage) {
  const int nj = -it.count;
  const int total = (int)it.begin;
  if (nj > kStageJobs || total > kStageElems) return;   // the planner never makes such items
  {
    const int32_t *s = reinterpret_cast<const int32_t *>(jobs + it.job);
    int32_t *d = reinterpret_cast<int32_t *>(Js);
    for (int w = threadIdx.x; w < nj * 32; w += kThreads) d[w] = s[w];
  }
  __syncthreads();
  const bool src_linear = Js[0].mode == 2;
  // load: contiguous source ranges (mode 2) or the strided source in its own order (mode 3)
  int j = 0;
  for (int e = threadIdx.x; e < total; e += kThreads) {
    while (j + 1 < nj && Js[j + 1].p <= e) j++;
    const CopyJob &J = Js[j];
    const int l = e - J.p;
    if (src_linear) {
      stage[e] = __ldg(src + J.src_off + l);
    } else {
      int64_t so, dof;
      staged_offsets(J, (uint32_t)l, so, dof);
      const int64_t at = J.p + dof;
      if (at < total) stage[at] = __ldg(src + J.src_off + so);
    }
  }
  __syncthreads();
  // store: the strided destination in its own order (mode 2) or contiguous ranges (mode 3)
  j = 0;
  for (int e = threadIdx.x; e < total; e += kThreads) {
    while (j + 1 < nj && Js[j + 1].p <= e) j++;
    const CopyJob &J = Js[j];
    const int l = e - J.p;
    if (src_linear) {
      int64_t so, dof;
      staged_offsets(J, (uint32_t)l, so, dof);
      const int64_t at = J.p + so;
      if (at < total) dst[J.dst_off + dof] = stage[at];
    } else {
      dst[J.dst_off + l] = stage[e];
    }
  }
}

__global__ void __launch_bounds__(kThreads) copy_kernel(const CopyJob *__restrict__ jobs,
                                                        const CopyItem *__restrict__ items,
                                                        const double *__restrict__ src,
                                                        double *__restrict__ dst) {
  __shared__ CopyJob Js[kStageJobs];
  __shared__ CopySmem sm;
  CopyJob &J = Js[0];
  auto &tile = sm.tile;
  const CopyItem it = items[blockIdx.x];
  if (it.count < 0) {
    copy_staged(jobs, it, src, dst, Js, sm.stage);
    return;
  }
  if (threadIdx.x < 32) {
    const int32_t *s = reinterpret_cast<const int32_t *>(&jobs[it.job]);
    reinterpret_cast<int32_t *>(&J)[threadIdx.x] = s[threadIdx.x];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nd = J.nd;
  if (J.mode == 0) {
    const int L = J.ext[nd - 1];
    const int64_t sin = J.sst[nd - 1];
    const int64_t din = J.dst[nd - 1];
    if (J.nchunk == 1 && L <= 16) {
      // several short rows per warp
      const int P = 32 / L;
      const int sub = lane / L, col = lane - sub * L;
      if (sub >= P) return;
      const int64_t end = it.begin + it.count;
      for (int64_t u = it.begin + (int64_t)warp * P + sub; u < end; u += (int64_t)kWarps * P) {
        int64_t so, dof;
        row_offsets(J, (uint32_t)u, so, dof);
        dst[dof + col * din] = src[so + col * sin];
      }
      return;
    }
    const int64_t end = it.begin + it.count;
    const uint32_t nchunk = (uint32_t)J.nchunk;
    for (int64_t u = it.begin + warp; u < end; u += kWarps) {
      const uint32_t row = (uint32_t)u / nchunk, chunk = (uint32_t)u - row * nchunk;
      int64_t so, dof;
      row_offsets(J, row, so, dof);
      const int c0 = (int)chunk * kRowChunk;
      const int n = min(kRowChunk, L - c0);
      so += c0 * sin;
      dof += c0 * din;
      if (sin == 1 && din == 1) {
        const double *s = src + so;
        double *d = dst + dof;
#pragma unroll 4
        for (int c = lane; c < n; c += 32) d[c] = __ldg(s + c);
      } else {
        for (int c = lane; c < n; c += 32) dst[dof + c * din] = src[so + c * sin];
      }
    }
    return;
  }
  // tile mode: q = nd-1 is destination-contiguous, p is source-contiguous
  const int q = nd - 1, p = J.p;
  const uint32_t ntq = (uint32_t)((J.ext[q] + kTile - 1) / kTile);
  const uint32_t ntp = (uint32_t)((J.ext[p] + kTile - 1) / kTile);
  const int64_t end = it.begin + it.count;
  for (int64_t u64 = it.begin; u64 < end; u64++) {
    uint32_t u = (uint32_t)u64;
    const uint32_t tq = u % ntq;
    u /= ntq;
    const uint32_t tp = u % ntp;
    u /= ntp;
    int64_t so = J.src_off, dof = J.dst_off;
    for (int i = nd - 1; i >= 0; i--) {
      if (i == p || i == q) continue;
      const uint32_t e = (uint32_t)J.ext[i];
      const uint32_t idx = u % e;
      u /= e;
      so += (int64_t)idx * J.sst[i];
      dof += (int64_t)idx * J.dst[i];
    }
    const int ep = J.ext[p], eq = J.ext[q];
    const int p0 = (int)tp * kTile, q0 = (int)tq * kTile;
    for (int i = warp; i < kTile; i += kWarps) {
      const int qq = q0 + i, pp = p0 + lane;
      if (qq < eq && pp < ep) tile[i][lane] = __ldg(src + so + pp + (int64_t)qq * J.sst[q]);
    }
    __syncthreads();
    for (int i = warp; i < kTile; i += kWarps) {
      const int pp = p0 + i, qq = q0 + lane;
      if (pp < ep && qq < eq) dst[dof + (int64_t)pp * J.dst[p] + qq] = tile[lane][i];
    }
    __syncthreads();
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

}  // namespace

cudaError_t launch_copy(const CopyJob *jobs, const CopyItem *items, int64_t nitems, const double *src,
                        double *dst, cudaStream_t stream) {
  if (nitems <= 0) return cudaSuccess;
  if (nitems > INT32_MAX) return cudaErrorInvalidValue;
  copy_kernel<<<(unsigned)nitems, kThreads, 0, stream>>>(jobs, items, src, dst);
  return cudaGetLastError();
}

cudaError_t launch_trace(const TraceOut *outs, int64_t nout, const TraceContrib *contribs,
                         const double *src, double *dst, cudaStream_t stream) {
  if (nout <= 0) return cudaSuccess;
  if (nout > INT32_MAX) return cudaErrorInvalidValue;
  trace_kernel<<<(unsigned)nout, 128, 0, stream>>>(outs, contribs, src, dst);
  return cudaGetLastError();
}

}  // namespace ytn
