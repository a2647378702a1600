// Launchers of the device kernels (copy_kernels.cu, gemm_fp64.cu, gemm_split.cu).
#pragma once

#include <cuda_runtime.h>

#include "ytn_internal.hpp"

namespace ytn {

// Move blocks between layouts: items[0..nitems) of the job table, src -> dst.
// max_nd: the most dims any of these items has (kind & 255); at most 4 selects the
// kernel with fewer registers.
cudaError_t launch_copy(const CopyJob *jobs, const CopyItem *items, int64_t nitems, const double *src,
                        double *dst, cudaStream_t stream, int max_nd = kMaxCopyDims);

// Trace: one CTA per output block.
cudaError_t launch_trace(const TraceOut *outs, int64_t nout, const TraceContrib *contribs,
                         const double *src, double *dst, cudaStream_t stream);

// Scalar product <A, B> over the planned common elements (FP64, deterministic):
// one partial per chunk into `partials`, then their fixed-order sum into out[0].
cudaError_t launch_vdot(const VdotChunk *chunks, int64_t nchunks, const VdotPiece *pieces, const double *a,
                        const double *b, double *partials, double *out, bool complex_data, cudaStream_t stream);

// Grouped FP64 GEMM (DMMA) over 64x64 tiles: C_q = A_q B_q.
cudaError_t launch_gemm_fp64(const SectorDev *sectors, const GemmTile *tiles, int64_t ntiles,
                             const double *wa, const double *wb, double *wc, cudaStream_t stream);

// Split-precision path: row exponents and BF16 slices of every sector operand.
// Staged path (from the FP64 sector matrices wa, wb): row exponents (ea, eb;
// emax[op] receives each operand's largest), then the slices.
cudaError_t launch_split_prep(const SplitOperand *ops, const SplitItem *exp_items, int64_t nexp,
                              const SplitItem *slice_items, int64_t nslice, const double *wa, const double *wb,
                              int32_t *ea, int32_t *eb, int32_t *emax, uint8_t *sa, uint8_t *sb, int slices,
                              cudaStream_t stream);

// Fused path: row exponents, then slices, straight from the tensors' blocks (a, b:
// the operands' data), two passes over the blocks, for the items [items, items +
// nitems). beside_gemm: the digits kernel sized to share each SM with a
// split-GEMM CTA (pipelined variant).
cudaError_t launch_split_blocks(const SplitOperand *ops, const SliceItem *items, int64_t nitems,
                                const SliceSeg *segs, const double *a, const double *b, int32_t *ea, int32_t *eb,
                                int32_t *emax, uint8_t *sa, uint8_t *sb, int slices, bool beside_gemm,
                                cudaStream_t stream);

// Shared-memory opt-in of the split-precision GEMM kernels (once per device).
cudaError_t configure_split_gemm();
// Shared-memory carveout of the slicing kernels that run beside the split GEMM.
cudaError_t configure_split_blocks();

// Scatter-combine of complex products: C blocks (interleaved complex) from the
// quadrants of the doubled real C_q (one CTA per job).
cudaError_t launch_cscatter(const CScatterJob *jobs, int64_t njobs, const double *wc, double *c,
                            cudaStream_t stream);

// N(0, 1) numbers: Philox4x32-10 words turned by Box-Muller (see ytn_fill_normal).
cudaError_t launch_fill_normal(uint64_t seed, int64_t n, double *out, cudaStream_t stream);

// Split-precision grouped GEMM (tcgen05) over 128x128 tiles (and 128x64 tiles
// when mixed_widths: the tile list holds them), FP64 output C_q;
// the epilogue adds each sector's scaled ||C_q||^2 into normsq (emax: the
// operands' largest exponents).
cudaError_t launch_gemm_split(const SplitSector *sectors, const SplitTile *tiles, int64_t ntiles, const uint8_t *sa,
                              const uint8_t *sb, const int32_t *ea, const int32_t *eb, const int32_t *emax,
                              float *normsq, double *wc, int slices, int *status, int num_sms, bool mixed_widths,
                              cudaStream_t stream);

// Accuracy check of the split products (one CTA per sector, the last one
// finalises): per-sector estimates from the exponents and normsq, the list of
// sectors above rtol with their 64 x 64 tile counts, the call's record, and the
// status word's tolerance flag (status[1]) when the fallback cannot reach rtol.
// eta_split / eta_fp64: per-element error of the split / FP64 products relative
// to the row and column scales, per square root of K.
cudaError_t launch_split_check(const SplitSector *sectors, int64_t nsec, const int32_t *ea, const int32_t *eb,
                               const int32_t *emax, const float *normsq, double *secv, int32_t *flagged,
                               int32_t *tile_end, int32_t *item_end_a, int32_t *item_end_b, SplitRecord *rec,
                               double eta_split, double eta_fp64, double rtol, int slices, int *status,
                               cudaStream_t stream);

// FP64 fallback of the fused split path: zero fill (partially populated
// operands) and gathers of the flagged sectors' FP64 sector matrices only
// (persistent grids over the flagged sectors' work items; item_end: running item
// counts per flagged sector, written by the accuracy check).
cudaError_t launch_gather_flagged(const CopyJob *jobs, const CopyItem *items_a, const CopyItem *items_b,
                                  const SplitSector *sp_sectors, const SectorDev *sectors, const int32_t *flagged,
                                  const int32_t *item_end_a, const int32_t *item_end_b, const SplitRecord *rec,
                                  const double *a, const double *b, double *wa, double *wb, bool zero_a, bool zero_b,
                                  int num_sms, cudaStream_t stream);

// FP64 recomputation of the flagged sectors (persistent, 64 x 64 DMMA tiles):
// the sector list and tile counts come from the accuracy check on the device.
cudaError_t launch_gemm_fp64_redo(const SectorDev *sectors, const int32_t *flagged, const int32_t *tile_end,
                                  const SplitRecord *rec, const double *wa, const double *wb, double *wc,
                                  int num_sms, cudaStream_t stream);

}  // namespace ytn
