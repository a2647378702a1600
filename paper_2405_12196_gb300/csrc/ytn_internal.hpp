// Internal types shared by the host planner (planner.cpp) and the device code
// (api.cu, copy_kernels.cu, gemm_fp64.cu, gemm_split.cu). Not part of the ABI.
#pragma once

#include <array>
#include <atomic>
#include <cstdint>
#include <memory>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/ytn.h"

namespace ytn {

// ----------------------------------------------------------------------------
// Device job tables
// ----------------------------------------------------------------------------

constexpr int kMaxCopyDims = 8;

// One piece of a block moved between two layouts (gather into a sector
// matrix, scatter out of one, fuse, unfuse). Every block copy has one dense
// side: the block itself, a contiguous range in its tensor. The planner cuts
// a block into pieces of at most kStageElems elements that are contiguous on
// that side; a CTA stages the pieces of one work item whole in shared memory.
//   mode 2: the dense side is the source. The piece is read linearly and
//           written in destination order.
//   mode 3: the dense side is the destination. The piece is read in source
//           order and written linearly.
// Dims are listed outer -> inner in the order of the strided (global) side,
// which has stride 1 innermost when the layouts allow, right-aligned in the
// kMaxCopyDims slots (the nd used ones last, unit dims before them): gstr are
// the strided side's strides from g_off, lstr the dense side's strides from
// the piece's start (d_off in global memory, p in the item's staging buffer).
// mag / shf divide by ext: n / ext = (n + umulhi(n, mag)) >> shf for n < 2^31.
struct CopyJob {
  int64_t g_off;
  int64_t d_off;
  int32_t nd;
  int32_t mode;
  int32_t p;
  int32_t size;
  int32_t ext[kMaxCopyDims];
  int32_t gstr[kMaxCopyDims];
  int32_t lstr[kMaxCopyDims];
  uint32_t mag[kMaxCopyDims];
  uint8_t shf[kMaxCopyDims];
  int32_t negate;      // 1: written negated (swap-gate sign); 2: imaginary parts
                       // negated (odd source offsets of interleaved complex data)
  int32_t reserved[5];
};
static_assert(sizeof(CopyJob) == 192, "CopyJob layout");

constexpr int kStageElems = 4096; // elements per CTA work item
constexpr int kStageJobs = 32;    // pieces per CTA work item

// A run of consecutive jobs [job, job + njobs) of one mode, processed by one
// CTA; kind = nd | mode << 8 with nd the largest dimension count of its jobs.
struct CopyItem {
  int32_t job;
  int32_t njobs;
  int32_t total;
  int32_t kind;
};
static_assert(sizeof(CopyItem) == 16, "CopyItem layout");

// One charge sector of a contraction: C_q (M x N, row-major, ldc = N) =
// A_q (M x K) B_q (K x N). A_q is stored K-major (M rows of K, lda = K) when
// a_kmajor, else M-major (K rows of M, lda = M); B_q is stored K-major
// (N rows of K, ldb = K) when b_kmajor, else N-major (K rows of N, ldb = N).
struct SectorDev {
  int64_t a_off, b_off, c_off;     // element offsets in the FP64 workspaces
  int32_t M, N, K;
  int32_t a_kmajor, b_kmajor;
  int32_t pad;
};
static_assert(sizeof(SectorDev) == 48, "SectorDev layout");

// One output tile of the grouped FP64 GEMM.
struct GemmTile {
  int32_t sector;
  int32_t mt, nt;   // tile coordinates in units of `size`
  int32_t size;     // tile edge: 64, or 32 for small sectors
};

// Trace: one output block, fed by ncontrib contributing input blocks.
struct TraceOut {
  int64_t dst_off;
  int32_t nrest;          // elements of the output block
  int32_t nrd;            // rest dims
  int32_t first, ncontrib;
  int32_t rext[kMaxCopyDims];
};
struct TraceContrib {
  int64_t src_off;
  int32_t ndiag;          // paired dims
  int32_t pad;
  int32_t rstr[kMaxCopyDims];   // input strides of the rest dims
  int32_t dext[kMaxCopyDims];   // extents of the paired dims
  int32_t dstr[kMaxCopyDims];   // sum of the two strides of each pair
};

// Scalar product: a contiguous run of elements common to A and B (part of one
// block, at most kVdotPiece elements), and a CTA's share: pieces
// [first, first + count) of the piece table.
constexpr int kVdotPiece = 4096;
constexpr int kVdotChunk = 8192;   // elements per CTA
struct VdotPiece {
  int64_t a_off, b_off;
  int32_t len, pad;
};
static_assert(sizeof(VdotPiece) == 24, "VdotPiece layout");
struct VdotChunk {
  int32_t first, count;
};

// ----------------------------------------------------------------------------
// Split-precision path tables
// ----------------------------------------------------------------------------

// Slices of one operand of one sector are stored pre-tiled and pre-swizzled:
// block (row tile rt of 128 rows, K stage kt of 32) holds kSlices slices of
// 128 x 32 BF16 each (8 KB per slice, the 64-byte-swizzled K-major layout the
// tensor cores read), so that one bulk copy moves a whole stage.
constexpr int kSplitBM = 128;              // rows per tile (M, and N)
constexpr int kSplitBK = 32;               // K per stage
constexpr int kSlices = 6;                 // slices stored per operand
constexpr int kSliceBytes = kSplitBM * kSplitBK * 2;         // 8192
constexpr int kBlockBytes = kSlices * kSliceBytes;           // 49152

// One operand (A rows = M, or B rows = N) of one sector, for the split kernels.
struct SplitOperand {
  int64_t src_off;     // element offset of the FP64 sector matrix in its workspace
  int64_t exp_off;     // int offset of its row exponents
  int64_t slice_off;   // byte offset of its slice blocks
  int32_t rows, K, ks, kmajor;   // kmajor: stored rows x K (ld = K), else K x rows
};
static_assert(sizeof(SplitOperand) == 40, "SplitOperand layout");

// Fused split (split_blocks.cu): the slices of an operand are built straight from
// the tensor's blocks. A work item covers 32 rows (a quarter of a 128-row tile)
// and 128 of K (four K stages); its segments are the parts of the blocks that
// fall inside it. Element (r, k) of a segment (r0 <= r < r1, k0 <= k < k1,
// item-relative) is the block's element (i, x) with i = ibase + r - r0 over the
// free dims fext (row-major) and x = kbase + k - k0 over the contracted dims kext,
// at boff + sum_d i_d fst_d + sum_d x_d kst_d doubles into the tensor's data.
// A segment is walked with the lanes along the block's contiguous direction
// (rfast: lanes are rows and the walk steps along K; else lanes are K, four per
// lane, and the walk steps along rows). Its cost is the number of warp-wide copy
// steps: k1 - k0 when rfast, else (r1 - r0) * ceil((k1 - k0) / 32). cost0: the
// summed cost of the item's segments before it; the loader gives each warp an
// equal share of the item's total cost (SliceItem::cost), cutting segments along
// their stepped direction.
constexpr int kSegDims = 4;       // dims per side in the table
constexpr int kFusedDims = 3;     // dims per side the planner puts on the fused path
constexpr int kItemRows = 32;     // rows per fused work item
constexpr int kItemK = 128;       // K per fused work item
constexpr int kPipeGroups = 8;    // most sector groups of the pipelined fused split
struct SliceSeg {
  int64_t boff;
  int64_t fst[kSegDims], kst[kSegDims];
  int32_t fext[kSegDims], kext[kSegDims];
  int32_t ibase, kbase;
  int32_t cost0;
  uint8_t pad0, nf, nk, rfast;
  int16_t r0, r1, k0, k1;
};
static_assert(sizeof(SliceSeg) == 128, "SliceSeg layout");

struct SliceItem {
  int32_t op, rt, quarter, kq;  // 128-row tile rt, its 32-row quarter; K from 128 kq
  int32_t seg0, nseg;
  int32_t full;                 // the segments cover every element (no zero fill)
  int32_t cost;                 // summed cost of the segments (warp-wide copy steps)
};
static_assert(sizeof(SliceItem) == 32, "SliceItem layout");

// Work item of the exponent / slicing kernels: operand, row tile, stage range.
struct SplitItem {
  int32_t op, rt, kt0, nkt;
};

struct SplitSector {
  int64_t sa_off, sb_off;    // byte offsets of the slice blocks of A and B
  int64_t ea_off, eb_off;    // int offsets of the row exponents of A and the column exponents of B
  int64_t c_off;             // element offset of C_q in the FP64 workspace
  int32_t M, N, K, ks;
  int32_t ga0, ga1, gb0, gb1; // the sector's gather items of A and B (FP64 fallback)
};
static_assert(sizeof(SplitSector) == 72, "SplitSector layout");

// One output tile of the split GEMM: 128 rows x bn columns (bn = 128, or 64 for a
// narrow tile; nt counts tiles of that width).
struct SplitTile {
  int32_t sector, mt, nt, bn;
};

// Accuracy check of a split-precision call, written into the workspace after the
// column exponents (see split_check.cu):
//   emax    int32 [2 * nsec]  largest row exponent of each operand (A of sector q
//                             at 2q, B at 2q + 1), max-combined by the exponent kernel
//   normsq  float [nsec]      ||C_q||_F^2 times 4^-(emax_A + emax_B), summed by the
//                             GEMM epilogue
//   SplitRecord               the call's totals (below)
//   secv    double [nsec]     K_q sum_i 4^(e_i - emax_A) sum_j 4^(f_j - emax_B)
//   flagged int32 [nsec]      sectors recomputed on the FP64 path, in sector order
//   tile_end int32 [nsec]     running count of their 64 x 64 FP64 tiles
// emax is filled with bytes 0x80 and normsq / the record with zeros before the
// call's kernels run.
struct SplitRecord {
  double err_est;          // relative Frobenius error of C after the FP64 fallback
  double split_err_est;    // the same for the split products alone (no fallback)
  double max_sector_est;   // largest per-sector estimate of the split products
  double fallback_flops;   // useful FLOPs recomputed on the FP64 path
  double rtol;             // tolerance the call was made with
  int32_t nsectors;
  int32_t nfallback;       // sectors recomputed on the FP64 path
  int32_t within;          // 1 when err_est <= rtol
  int32_t valid;           // 1 once the check has run
  int32_t done_blocks;     // per-sector CTAs finished (the last one finalises)
  int32_t slices;
};
static_assert(sizeof(SplitRecord) == 64, "SplitRecord layout");

// Scatter of a complex product: one C block from the quadrants of the doubled
// C_q (P = [[re.re, re.im], [im.re, im.im]] in rows x columns): element e of the
// block (row-major over its nd dims) reads P at src + sum idx_i sstr_i plus the
// quadrant offsets q01, q10, q11 (-1: quadrant absent, a real operand), and
// writes re = P00 - P11, im = P01 + P10 at complex element dst + e.
struct CScatterJob {
  int64_t src, dst;
  int64_t q01, q10, q11;
  int32_t nd, n;
  int32_t ext[kMaxCopyDims];
  int64_t sstr[kMaxCopyDims];
};

// ----------------------------------------------------------------------------
// Host-side structures
// ----------------------------------------------------------------------------

struct Fusion {
  int nlegs = 0;
  int sig[YTN_MAX_RANK] = {0};
  int64_t nentries = 0;
  std::vector<int32_t> nu;   // [nentries][nsym]
  std::vector<int32_t> t;    // [nentries][nlegs][nsym]
  std::vector<int64_t> D;    // [nentries][nlegs]
};

struct Tensor {
  int dtype = YTN_REAL64;    // YTN_COMPLEX128: elements are (re, im) pairs of doubles
  int nsym = 0;
  int mod[YTN_MAX_SYM] = {0};
  int rank = 0;
  int sig[YTN_MAX_RANK] = {0};
  int n[YTN_MAX_SYM] = {0};
  int64_t nblocks = 0;
  std::vector<int32_t> t;    // [nblocks][rank][nsym]
  std::vector<int64_t> D;    // [nblocks][rank]
  std::vector<int64_t> off;  // [nblocks]
  // [nblocks][rank] element strides of each block; empty = row-major blocks.
  // Only planner-internal views (a fused leg seen as its constituents) set it.
  std::vector<int64_t> bstr;
  int64_t size = 0;
  std::shared_ptr<Fusion> fus[YTN_MAX_RANK];

  const int32_t *charge(int64_t b, int leg) const { return &t[((size_t)b * rank + leg) * nsym]; }
  int64_t dim(int64_t b, int leg) const { return D[(size_t)b * rank + leg]; }
  int64_t elems(int64_t b) const {
    int64_t e = 1;
    for (int i = 0; i < rank; i++) e *= dim(b, i);
    return e;
  }
};

struct HostSector {
  int64_t M = 0, N = 0, K = 0;
  int64_t a_off = 0, b_off = 0, c_off = 0;
};

enum class Kind { Tensordot = 1, Fuse = 2, Unfuse = 3, Trace = 4, Vdot = 5, Swap = 6, Conj = 7, Svd = 8, Slice = 9,
                  Eigh = 10, Blocks = 11 };

// One charge sector of a block-diagonal SVD: the dense m x n matrix M and where
// its factors live in the workspace (offsets in doubles). The solver factors a
// column-major X with at least as many rows as columns: X = M^T (M stored
// row-major) when n >= m, else X = M (stored column-major; trans = 1). Either
// way M = F_m diag(S) F_n^T with F_m (m x k) and F_n (n x k) column-major.
struct SvdSector {
  int64_t m, n, k, trans;
  int64_t m_off, up_off, vp_off;   // X, F_n, F_m: offsets in elements (complex: pairs)
  int64_t s_off;                   // S (real): offset in doubles
};

struct Plan;

}  // namespace ytn

struct ytn_ctx {
  int device = 0;
  int *status_dev = nullptr;   // device status word (bounded waits report here)
  int num_sms = 0;
  std::atomic<int> gemm_sms{0};   // CTAs of the persistent split GEMM (0: one per SM)
  std::mutex mu;
  std::unordered_map<std::string, ytn_plan_t *> cache;
  // phase timing: a pool of CUDA events (cudaEvent_t stored as void*) and the
  // (phase, start-event index) pairs recorded since the last read
  bool prof = false;
  std::vector<void *> ev_pool;
  size_t ev_next = 0;
  std::vector<std::pair<int, int>> pending;
  int64_t dropped = 0;
  std::mutex prof_mu;
  // graph capture: the stream being captured (cudaStream_t as void*) and the
  // plans whose device tables the recorded launches use (one reference each)
  std::atomic<bool> capturing{false};
  void *cap_stream = nullptr;
  std::vector<ytn_plan_s *> cap_plans;
  std::mutex cap_mu;
  // dense solver: kSolverLanes handles, parameter sets, streams and events
  // (created by the first SVD / eigh plan); sectors are factored concurrently
  std::vector<void *> solvers, solver_params, solver_streams, solver_events;
  std::mutex solver_mu;
  // pipelined fused split: the GEMM chain's stream (highest priority), the
  // slicing stream (lowest) and their events (created with the context); one
  // call's enqueue at a time
  void *pipe_hi = nullptr, *pipe_lo = nullptr;
  std::vector<void *> pipe_ev;
  std::mutex pipe_mu;
};

struct ytn_plan_s {
  std::atomic<int> refs{1};
  ytn_ctx *ctx = nullptr;
  ytn::Kind kind = ytn::Kind::Tensordot;
  std::string key;
  // tensordot shard (ytn_plan_shard): this plan keeps the work units that the
  // partition of the whole contraction over shard_world ranks gives shard_rank
  int32_t shard_rank = 0, shard_world = 1;

  // input sizes and output structure (owned storage + ABI view)
  int64_t a_size = 0, b_size = 0;
  int ca = 1, cb = 1;   // tensordot: 2 when A (B) is complex (doubled sector matrices)
  // further outputs (SVD: S and V after U in `out`) and their ABI views
  std::vector<ytn::Tensor> outs;
  std::vector<ytn_struct> outs_view;
  std::vector<std::vector<ytn_fusion>> outs_fus_view;
  // SVD: sectors, the copy-item ranges of the output scatters, workspace layout
  std::vector<ytn::SvdSector> svd_sec;
  int64_t items_s_begin = 0, items_s_end = 0;   // S vectors -> S diagonals
  int64_t items_h_begin = 0, items_h_end = 0;   // complex: conjugate one factor in place
  size_t svd_m_doubles = 0, svd_ws_doubles = 0, svd_info_off = 0, svd_lwork = 0;
  std::vector<std::vector<char>> svd_host_ws;   // the solver's host buffer, per lane
  bool svd_zero_m = false;
  // doubles per element of the copy jobs that add_copy makes: 2 for complex
  // tensors moved whole (fuse, unfuse, swap gate, conj), else 1
  int cw = 1;
  ytn::Tensor out;
  ytn_struct out_view{};
  std::vector<ytn_fusion> out_fus_view;

  // tensordot
  std::vector<ytn::HostSector> sectors;
  std::vector<ytn::SectorDev> sectors_dev;
  std::vector<ytn::GemmTile> tiles;
  bool zero_a = false, zero_b = false;
  bool a_kmajor = true, b_kmajor = false;
  int64_t a_elems = 0, b_elems = 0, c_elems = 0;
  int64_t max_m = 0, max_n = 0, max_k = 0;
  double flops = 0;

  // data movers: all copy jobs, and item ranges per phase
  std::vector<ytn::CopyJob> jobs;
  std::vector<ytn::CopyItem> items;
  int64_t items_a_begin = 0, items_a_end = 0;   // gather A (tensordot) or the single phase
  int64_t items_b_begin = 0, items_b_end = 0;   // gather B
  int64_t items_c_begin = 0, items_c_end = 0;   // scatter C
  bool zero_out = false;                        // fuse: output needs zero fill
  int64_t moved = 0;

  // trace
  std::vector<ytn::TraceOut> tr_out;
  std::vector<ytn::CScatterJob> cs_jobs;   // complex tensordot: the scatter-combine
  std::vector<ytn::TraceContrib> tr_contrib;
  std::vector<ytn::VdotPiece> vd_pieces;
  std::vector<ytn::VdotChunk> vd_chunks;

  // device copies of the tables (one allocation)
  void *dev = nullptr;
  size_t dev_bytes = 0;
  const ytn::CopyJob *d_jobs = nullptr;
  const ytn::CopyItem *d_items = nullptr;
  const ytn::SectorDev *d_sectors = nullptr;
  const ytn::GemmTile *d_tiles = nullptr;
  const ytn::TraceOut *d_tr_out = nullptr;
  const ytn::CScatterJob *d_cs_jobs = nullptr;
  const ytn::TraceContrib *d_tr_contrib = nullptr;
  const ytn::VdotPiece *d_vd_pieces = nullptr;
  const ytn::VdotChunk *d_vd_chunks = nullptr;

  // split-precision tables
  std::vector<ytn::SplitOperand> sp_ops;
  std::vector<ytn::SplitItem> sp_exp_items, sp_slice_items;
  // fused split: items and segments (empty when a block has more than kSegDims
  // free or contracted dims: then the staged path gathers first); the tensor
  // blocks behind them, recorded while the gathers are planned
  std::vector<ytn::SliceItem> sp_fitems;
  std::vector<ytn::SliceSeg> sp_segs;
  bool sp_fused = false;
  // pipelined fused split: the sectors in the GEMM's order cut into groups; per
  // group the end of its tiles in sp_tiles and of its items in sp_fitems (empty:
  // fewer than two groups). Group g's slicing runs beside group g - 1's GEMM.
  std::vector<int64_t> sp_pipe_tile_end, sp_pipe_item_end;
  std::vector<std::array<int64_t, 4>> sec_gather_items;   // per sector: A items, B items (relative)
  std::vector<ytn::SplitSector> sp_sectors;
  std::vector<ytn::SplitTile> sp_tiles;
  std::vector<ytn::SplitTile> sp_tiles_mix;    // with 64-wide sector tails (empty: none)
  int64_t sp_sa_bytes = 0, sp_sb_bytes = 0, sp_ea = 0, sp_eb = 0;
  // YTN_AUTO: per slice count, -1 undecided, 0 FP64, 1 split; the timings (ms)
  std::mutex auto_mu;
  int auto_choice[ytn::kSlices + 1] = {-1, -1, -1, -1, -1, -1, -1};
  float auto_ms[ytn::kSlices + 1][2] = {};
  // split path variant per slice count: -1 undecided, 0 staged, 1 fused (slices
  // straight from the blocks), 2 fused and pipelined with the GEMM; the timings
  // (ms) of the three
  int split_variant[ytn::kSlices + 1] = {-1, -1, -1, -1, -1, -1, -1};
  float variant_ms[ytn::kSlices + 1][3] = {};
  // split GEMM tile list per slice count: -1 undecided, 0 all 128 wide, 1 with the
  // 64-wide sector tails; the timings (ms)
  int tile_policy[ytn::kSlices + 1] = {-1, -1, -1, -1, -1, -1, -1};
  float tile_ms[ytn::kSlices + 1][2] = {};
  const ytn::SliceItem *d_sp_fitems = nullptr;
  const ytn::SliceSeg *d_sp_segs = nullptr;
  const ytn::SplitOperand *d_sp_ops = nullptr;
  const ytn::SplitItem *d_sp_exp_items = nullptr, *d_sp_slice_items = nullptr;
  const ytn::SplitSector *d_sp_sectors = nullptr;
  const ytn::SplitTile *d_sp_tiles = nullptr, *d_sp_tiles_mix = nullptr;
  // the most dims of any copy item in a range [begin, end) of `items` (selects the
  // copy kernel built for at most 4 dims), computed on first use
  std::mutex nd_mu;
  std::unordered_map<int64_t, int> nd_max;   // key: begin * 2^32 + end
};

namespace ytn {

// planner.cpp
ytn_status load_struct(const ytn_struct *s, Tensor &T, std::string &err);
ytn_status plan_tensordot(ytn_plan_t *p, const Tensor &A, const Tensor &B, int naxes,
                          const int *axa, const int *axb, std::string &err);
ytn_status plan_fuse(ytn_plan_t *p, const Tensor &A, int ngroups, const int *group_size,
                     const int *order, std::string &err);
ytn_status plan_unfuse(ytn_plan_t *p, const Tensor &A, int naxes, const int *axes,
                       std::string &err);
ytn_status plan_vdot(ytn_plan_t *p, const Tensor &A, const Tensor &B, std::string &err);
ytn_status plan_swap_gate(ytn_plan_t *p, const Tensor &A, int ngroups, const int *group_size, const int *order,
                          uint32_t fermionic, std::string &err);
ytn_status plan_conj(ytn_plan_t *p, const Tensor &A, std::string &err);
ytn_status plan_svd(ytn_plan_t *p, const Tensor &A, int ngroups, const int *group_size, const int *order,
                    std::string &err);
ytn_status plan_eigh(ytn_plan_t *p, const Tensor &A, int ngroups, const int *group_size, const int *order,
                     std::string &err);
ytn_status plan_blocks(ytn_plan_t *p, const ytn_sym &sym, int rank, const ytn_leg *legs, const int32_t *n,
                       std::string &err);
ytn_status plan_slice(ytn_plan_t *p, const Tensor &A, int naxes, const int *axes, int64_t nkeep,
                      const int32_t *keep_t, const int64_t *keep_D, std::string &err);
void make_view(const Tensor &C, ytn_struct &v, std::vector<ytn_fusion> &fv);
ytn_status plan_trace(ytn_plan_t *p, const Tensor &A, int naxes, const int *ax1,
                      const int *ax2, std::string &err);
std::string plan_key(const ytn_op *op);
void finish_output_view(ytn_plan_t *p);
// Where one block of an operand lands in its sector matrix (rows: A's rows or
// B's columns; K), with the block's free and contracted dims and their strides in
// doubles (complex data: one entry per component).
struct SegSource {
  int64_t sector = 0, roff = 0, rlen = 0, koff = 0, klen = 0, boff = 0;
  std::vector<int64_t> fext, fst, kext, kst;
};
void plan_split_tables(ytn_plan_t *p, std::vector<SegSource> *src);

// error reporting (api.cu)
ytn_status fail(ytn_status st, const std::string &msg);

// dense solver of the block-diagonal SVD (svd.cpp): sectors are factored on
// kSolverLanes handles and streams at once, each with its own device buffer
constexpr int kSolverLanes = 8;
ytn_status svd_prepare(ytn_plan_t *p);
ytn_status svd_factor(ytn_plan_t *p, double *ws, void *stream);
void svd_release(ytn_ctx *ctx);

}  // namespace ytn
