// Launchers of the device kernels (copy_kernels.cu, gemm_fp64.cu, gemm_split.cu).
#pragma once

#include <cuda_runtime.h>

#include "ytn_internal.hpp"

namespace ytn {

// Move blocks between layouts: items[0..nitems) of the job table, src -> dst.
cudaError_t launch_copy(const CopyJob *jobs, const CopyItem *items, int64_t nitems, const double *src,
                        double *dst, cudaStream_t stream);

// Trace: one CTA per output block.
cudaError_t launch_trace(const TraceOut *outs, int64_t nout, const TraceContrib *contribs,
                         const double *src, double *dst, cudaStream_t stream);

// Grouped FP64 GEMM (DMMA) over 64x64 tiles: C_q = A_q B_q.
cudaError_t launch_gemm_fp64(const SectorDev *sectors, const GemmTile *tiles, int64_t ntiles,
                             const double *wa, const double *wb, double *wc, cudaStream_t stream);

}  // namespace ytn
