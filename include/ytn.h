/*
 * ytn.h -- C ABI of a single-GPU (GB300, sm_103a) library that contracts
 * abelian-symmetric block-sparse tensors.
 *
 * The operations follow "YASTN: Yet another symmetric tensor networks"
 * (arXiv 2405.12196):
 *   - Sec. II.A: a leg V(s, t, D) has a signature s = +-1, charge sectors t and
 *     their dimensions D; a rank-N tensor stores dense blocks keyed by one
 *     sector per leg, and a stored block (rho_1..rho_N) satisfies
 *     sum_i s_i rho_i = n (block form of Eq. elemchargecon). Charges of U(1) are
 *     integers, of Z_m integers modulo m, of product groups tuples of these.
 *   - Sec. II.A (storage): blocks are serialised into one 1-D array.
 *   - Sec. II.B: fusion of legs (fused charge nu = s_r (s_i rho + s_j rho'),
 *     fused dimension D_nu = sum D_rho D_rho'), its inverse (unfusion, from the
 *     recorded original structure), and contraction = fuse into matrices,
 *     multiply per charge sector, unfuse (the contraction equation), with the
 *     non-zero blocks precomputed before any dense work.
 *
 * Model of use: describe the tensors' block structure on the host (ytn_struct),
 * call ytn_plan once per structure (pure host integer work plus one upload of
 * job tables to the device; cached), then run the plan on device data as often
 * as needed (ytn_tensordot / ytn_fuse / ytn_unfuse / ytn_trace). Execution
 * calls are asynchronous on the given stream and allocate nothing.
 *
 * Conventions for every tensor in this API
 *   - data are FP64, one device buffer per tensor; block b occupies
 *     [off[b], off[b] + prod_i D[b][i]) of it, row-major (C order);
 *   - blocks are listed in canonical order: strictly ascending lexicographic
 *     order of the flattened (rank x nsym) charge tuple;
 *   - Z_m charge components are given reduced, in [0, m).
 *
 * Ownership
 *   - every host array passed in (ytn_struct, ytn_fusion) belongs to the
 *     caller and is read only during the call; the plan keeps its own copies;
 *   - plans and the output structure they describe belong to the library
 *     (release with ytn_plan_release);
 *   - device buffers (inputs, outputs, workspace) belong to the caller.
 *
 * Errors: every call returns a ytn_status; nothing is thrown across the ABI.
 * Structural errors are found by ytn_plan, before any device work. A short
 * message for the last error of the calling thread is in ytn_last_error().
 */
#ifndef YTN_H
#define YTN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define YTN_MAX_RANK 16
#define YTN_MAX_SYM 4

typedef enum {
  YTN_OK = 0,
  YTN_E_INVALID = 1,          /* malformed descriptor, axes, order or sizes      */
  YTN_E_SIGNATURE = 2,        /* contracted/traced legs with equal signatures    */
  YTN_E_DIM_MISMATCH = 3,     /* one charge with two dimensions on paired legs   */
  YTN_E_FUSION_MISMATCH = 4,  /* contracted fused legs with different histories  */
  YTN_E_NOMEM = 5,            /* host or device allocation failed                */
  YTN_E_CUDA = 6,             /* a CUDA runtime call failed                      */
  YTN_E_TIMEOUT = 7,          /* a bounded device wait ran out                   */
  YTN_E_UNSUPPORTED = 8,      /* valid request outside what this build handles   */
  YTN_E_TOLERANCE = 9,        /* requested accuracy cannot be guaranteed         */
  YTN_E_CHARGE = 10,          /* a block violates charge conservation            */
  YTN_E_WORKSPACE = 11        /* workspace missing or too small                  */
} ytn_status;

typedef enum {
  YTN_FP64 = 0,        /* FP64 operands, FP64 tensor-core (DMMA) products        */
  YTN_SPLIT_BF16 = 1,  /* FP64 operands split into BF16 slices, tcgen05 products  *
                        * with exact FP32 accumulation, recombined to FP64        */
  YTN_AUTO = 2         /* the faster of the two for this plan among those that   *
                        * meet rtol (FP64 always does): autotuned, see            *
                        * ytn_tensordot                                           */
} ytn_precision;

/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st *ytn_stream;

typedef struct ytn_ctx ytn_ctx;
typedef struct ytn_plan_s ytn_plan_t;
typedef struct ytn_ncon_s ytn_ncon_t;

/* Abelian group: nsym components; mod[c] == 0 is U(1), mod[c] == m > 1 is Z_m. */
typedef struct {
  int32_t nsym;
  int32_t mod[YTN_MAX_SYM];
} ytn_sym;

/* What a fused leg remembers of its origin (Sec. II.B: "records the original
 * structure"). For each fused charge nu, in ascending order of nu, the
 * constituent charge tuples present in the tensor in ascending order, each
 * with its constituent dimensions; sub-block e of sector nu occupies
 * prod_i D[e][i] consecutive indices of the fused sector, row-major over the
 * constituent legs, after the sub-blocks listed before it. */
typedef struct {
  int32_t nlegs;              /* m: constituent legs (2..YTN_MAX_RANK)        */
  int8_t sig[YTN_MAX_RANK];   /* constituent signatures                       */
  int64_t nentries;           /* rows of the record                           */
  const int32_t *nu;          /* [nentries][nsym] fused charge of each row    */
  const int32_t *t;           /* [nentries][nlegs][nsym] constituent charges  */
  const int64_t *D;           /* [nentries][nlegs] constituent dimensions     */
} ytn_fusion;

/* Element type of a tensor's data buffer. YTN_COMPLEX128 elements are pairs of
 * doubles (real, imaginary), interleaved; offsets and sizes count elements. The
 * paper's backends hold real or complex blocks (Sec. II.A footnote on
 * conjugation of complex tensors). */
typedef enum { YTN_REAL64 = 0, YTN_COMPLEX128 = 1 } ytn_dtype;

/* Block structure of one tensor (host memory, caller-owned). */
typedef struct {
  ytn_sym sym;
  int32_t rank;               /* 0..YTN_MAX_RANK                              */
  int8_t sig[YTN_MAX_RANK];   /* leg signatures, +1 or -1                     */
  int32_t n[YTN_MAX_SYM];     /* total charge                                 */
  int64_t nblocks;
  const int32_t *t;           /* [nblocks][rank][nsym] block charges          */
  const int64_t *D;           /* [nblocks][rank] block dimensions (>= 1)      */
  const int64_t *off;         /* [nblocks] element offsets into the data
                                 buffer; NULL means packed in block order     */
  int64_t size;               /* elements in the data buffer                  */
  const ytn_fusion *fus[YTN_MAX_RANK]; /* per leg; NULL for a plain leg       */
  int32_t dtype;              /* ytn_dtype of the data (0 = real FP64)        */
} ytn_struct;

#define YTN_FERMIONIC_EXPLICIT 0x80000000u

typedef enum {
  YTN_OP_TENSORDOT = 1,  /* C = sum_x A B over pairs (axa[k], axb[k]), Sec. II.B */
  YTN_OP_FUSE = 2,       /* fuse groups of legs, Sec. II.B                        */
  YTN_OP_UNFUSE = 3,     /* undo the fusion of legs axa[0..naxes), Sec. II.B      */
  YTN_OP_TRACE = 4,      /* sum the diagonals of leg pairs (axa[k], axb[k]) of a  */
  YTN_OP_VDOT = 5,       /* scalar product <a, b> of two tensors on the same legs */
  YTN_OP_SWAP_GATE = 6,  /* fermionic swap gate between two groups of legs, Sec. IV */
  YTN_OP_CONJ = 7,       /* conjugate: signatures flip, elements conjugated       */
  YTN_OP_SVD = 8,        /* block-diagonal SVD: rows | columns, Sec. III (CTM)    */
  YTN_OP_SLICE = 9,      /* keep the first keep[c] indices of sectors of legs     */
  YTN_OP_EIGH = 10       /* block-diagonal Hermitian eigendecomposition           */
} ytn_op_kind;

/* A planned operation.
 *  TENSORDOT: a, b, naxes pairs (axa[k] of a, axb[k] of b). Output legs: the
 *             free legs of a in order, then those of b; n_C = n_A + n_B.
 *  FUSE:      a, ngroups groups; order[] lists the legs group by group
 *             (group g has group_size[g] legs); every leg exactly once. A
 *             group of one leg passes through; a group of >= 2 legs must
 *             consist of plain legs. The fused leg takes the signature of its
 *             group's first leg.
 *  UNFUSE:    a, naxes fused legs axa[]; each is replaced by its constituents.
 *  TRACE:     a, naxes pairs (axa[k], axb[k]) of legs of a, with opposite
 *             signatures (the paper has no trace; this is the block-diagonal
 *             sum that the block structure implies).
 *  VDOT:      a, b on the same legs: same symmetry, rank and signatures, one
 *             dimension per charge on each leg, identical fusion records. The
 *             output is one element (a rank-0 tensor).
 *  SWAP_GATE: a, ngroups = 2 groups of legs (group_size, order as for FUSE;
 *             disjoint, each leg at most once). A block changes sign when the
 *             parities of both groups' charges are odd (Sec. IV: the swap gate
 *             at a crossing of two lines in the fermionic order). The parity
 *             of a charge is the sum of its fermionic components modulo 2;
 *             `fermionic` selects them: 0 = every component; otherwise
 *             YTN_FERMIONIC_EXPLICIT | (bit c for component c), so that an
 *             explicit empty set (all components bosonic) is expressible. Each
 *             fermionic component must be U(1) or Z_m with m even. Output
 *             structure = a's.
 *  CONJ:      a. Sec. II.A footnote: every leg's signature flips (n becomes
 *             -n, fusion records' constituent signatures flip) and complex
 *             elements are conjugated; blocks keep their charges and places.
 *  SVD:       a (real or complex), ngroups = 2: the row legs, then the
 *             column legs (every leg once). Three outputs (ytn_plan_output_at 0, 1, 2): U on (row
 *             legs, new leg, signature -1), S on (new leg +1, new leg -1) with a
 *             k x k diagonal block per sector, V on (new leg +1, column legs);
 *             the new leg carries the signed sum c of the row charges, with
 *             k_c = min(rows, columns) of sector c. U S V = a.
 *  EIGH:      a (Hermitian), ngroups = 2: row legs, then column legs dual
 *             to them in the same order, n = 0. Two outputs: U (row legs,
 *             new leg -1) and S (new leg +1, new leg -1; diagonal eigenvalues
 *             per sector, ascending); a = U S U^H. The lower triangle of each
 *             sector matrix is read.
 *  SLICE:     a, naxes legs axa[]; nkeep rows of (keep_t[nsym] charge,
 *             keep_D dimension): every sector of those legs keeps its first
 *             keep_D indices (charges not listed keep 0: their blocks go).
 *             Truncation of U, S, V to the kept singular values. */
typedef struct {
  ytn_op_kind kind;
  const ytn_struct *a;
  const ytn_struct *b;
  int32_t naxes;
  int32_t axa[YTN_MAX_RANK];
  int32_t axb[YTN_MAX_RANK];
  int32_t ngroups;
  int32_t group_size[YTN_MAX_RANK];
  int32_t order[YTN_MAX_RANK];
  uint32_t fermionic;         /* SWAP_GATE only: 0 = all components fermionic, else
                                 YTN_FERMIONIC_EXPLICIT | component bits      */
  int64_t nkeep;              /* SLICE only: rows of the keep table           */
  const int32_t *keep_t;      /* SLICE: [nkeep][nsym] charges                 */
  const int64_t *keep_D;      /* SLICE: [nkeep] kept dimensions               */
} ytn_op;

/* Sizes of a plan. */
typedef struct {
  double useful_flops;       /* sum over matching block pairs of 2|I||x||J|     */
  int64_t nsectors;          /* charge sectors with at least one product        */
  int64_t max_m, max_n, max_k;
  int64_t a_elems, b_elems, c_elems; /* elements of the sector matrices        */
  int64_t moved_elems;       /* elements read (= written) by the data movers    */
  int64_t out_size;          /* elements of the output data buffer              */
  int64_t njobs;             /* copy jobs of all data movers                    */
  int32_t split_fused;       /* 1: the split path builds its BF16 slices straight
                                from the blocks (at most three dims per side in
                                every block once unit dims are dropped and
                                contiguous ones merged); 0: it gathers FP64
                                sector matrices first                          */
  int32_t max_copy_dims;     /* most dims of any piece of the plan's data movers
                                (after merging contiguous dims); up to 4 runs the
                                copy kernel built for four, more the one for eight */
  int32_t split_pipe_groups; /* sector groups of the pipelined fused split (see
                                ytn_tensordot), 0 when the plan has none       */
} ytn_plan_info;

/* Per-call result of ytn_tensordot, filled when the call returns (before the
 * device has run it). */
typedef struct {
  double useful_flops;
  int32_t precision;         /* ytn_precision used                              */
  int32_t slices;            /* split path: BF16 slices per operand, else 0     */
  double err_est;            /* split path: the a-priori forecast that picks the
                                slice count (the data-aware estimate for data
                                spread like a normal distribution); 0 for FP64.
                                The estimate of this result, computed on the
                                device from its data, is in ytn_tensordot_report */
  int32_t split_variant;     /* split path: 1 when the BF16 slices were built
                                straight from the blocks (fused), 2 the same
                                pipelined with the GEMM, 0 when FP64 sector
                                matrices were gathered first (staged); -1 for
                                FP64                                           */
  int32_t narrow_tiles;      /* split path: 1 when sectors whose N ends in the
                                first half of a 128-wide tile had a 64-wide last
                                column tile, else 0                            */
} ytn_result;

/* Accuracy record of a split-precision ytn_tensordot (no counterpart in the
 * paper), computed on the device by the call itself and read with
 * ytn_tensordot_report. Per charge sector q the split products are estimated to
 * be off, per element, by eta(s) sqrt(K_q) 2^(e_i + f_j), where 2^e_i and 2^f_j
 * are the power-of-two scales of row i of A_q and column j of B_q (the split's
 * own scales); the sector's relative Frobenius error is then
 *   est_q = eta(s) sqrt(K_q sum_i 4^e_i sum_j 4^f_j) / ||C_q||_F,
 * which grows when the result is small against the scales (cancellation, or
 * rows whose elements lie far below their largest). Every sector with
 * est_q > rtol is recomputed on the FP64 path in the same call, so each sector,
 * and the whole result, stays within rtol unless even FP64 cannot reach it. */
typedef struct {
  double err_est;            /* relative Frobenius error of C, after the FP64
                                recomputation of the flagged sectors            */
  double split_err_est;      /* the same for the split products alone           */
  double max_sector_est;     /* largest est_q of the split products             */
  double fallback_flops;     /* useful FLOPs recomputed on the FP64 path        */
  double rtol;               /* tolerance of the call                           */
  int32_t nsectors;
  int32_t nfallback;         /* sectors recomputed on the FP64 path             */
  int32_t within;            /* 1 when err_est <= rtol                          */
  int32_t slices;
} ytn_error_report;

/* Context bound to one CUDA device; allocates a device status word.
 * device < 0 creates a host-only context: ytn_plan then builds plans (output
 * structure, sizes, job tables) without uploading them, and the execution
 * calls on such plans return YTN_E_INVALID. */
ytn_status ytn_ctx_create(ytn_ctx **ctx, int device);
void ytn_ctx_destroy(ytn_ctx *ctx);

/* Plan an operation: validates the structures (conservation, canonical order,
 * one dimension per charge and leg, compatibility of paired legs), matches
 * blocks by charge, groups them into sectors, builds the output structure and
 * the job tables, and uploads the tables to the context's device (synchronous
 * cudaMalloc + copy). Plans are cached by the full integer structure and the
 * operation: an identical request returns the cached plan with one more
 * reference. Errors: YTN_E_INVALID, YTN_E_CHARGE, YTN_E_SIGNATURE,
 * YTN_E_DIM_MISMATCH, YTN_E_FUSION_MISMATCH, YTN_E_UNSUPPORTED, YTN_E_NOMEM,
 * YTN_E_CUDA. */
ytn_status ytn_plan(ytn_ctx *ctx, const ytn_op *op, ytn_plan_t **plan);

/* One rank's part of a contraction split over `world` ranks (a TENSORDOT op; no
 * counterpart in the paper). The charge sectors of a contraction are independent
 * matrix products and every block of C lies in exactly one sector (Sec. II.B), so
 * the sectors can be shared out with no exchange of data: the work units are
 * whole sectors, except that a sector above a quarter of a rank's share of the
 * useful FLOPs is cut into runs of consecutive row charge tuples I of about that
 * size; units go to ranks longest first, each to the least loaded rank (ties to
 * the lower rank, units of equal FLOPs in sector and row order). Every rank
 * computes the same partition from the structure alone. The plan is an ordinary
 * tensordot plan on the whole A and B (replicated on every rank) whose output
 * structure holds only this rank's blocks of C, in canonical order and packed;
 * the union over ranks of the output blocks is the output of ytn_plan for the
 * same op, with the same values. ytn_plan_get_info reports this rank's useful
 * FLOPs and sectors. world = 1 is ytn_plan. Plans are cached per (op, rank,
 * world). Errors: as ytn_plan, plus YTN_E_INVALID (rank outside [0, world), or
 * world > 1 for another kind of op). */
ytn_status ytn_plan_shard(ytn_ctx *ctx, const ytn_op *op, int32_t rank, int32_t world, ytn_plan_t **plan);

/* A leg V(s, t, D) (Sec. II.A): signature, and its charge sectors with their
 * dimensions, in ascending charge order. */
typedef struct {
  int8_t sig;
  int32_t ncharges;
  const int32_t *t;           /* [ncharges][nsym] */
  const int64_t *D;           /* [ncharges], >= 1 */
} ytn_leg;

/* The structure of a tensor on the given legs with total charge n (Sec. II.A,
 * the paper's rand(legs, n)): every block allowed by the conservation rule
 * sum_i s_i rho_i = n (modulo m for Z_m components), canonical order, packed.
 * The plan's output structure is that tensor; ytn_fill_normal fills its data.
 * Errors: YTN_E_INVALID (legs, charges), YTN_E_UNSUPPORTED (more than 2^31 blocks). */
ytn_status ytn_plan_blocks(ytn_ctx *ctx, ytn_sym sym, int32_t rank, const ytn_leg *legs, const int32_t *n,
                           ytn_plan_t **plan);

/* out (the plan's output size, real FP64; device or page-locked host memory) = N(0, 1)
 * numbers: element i is word i mod 4 of Philox4x32-10 (Salmon et al., SC'11) at
 * counter (i div 4, 0, 0) and key seed, each pair of words (x, y) turned by the
 * Box-Muller transform into sqrt(-2 ln u) (cos, sin)(2 pi v), u = (x + 1) 2^-32,
 * v = y 2^-32. Deterministic. Asynchronous on stream. */
ytn_status ytn_fill_normal(ytn_plan_t *plan, uint64_t seed, double *out, ytn_stream stream);

/* Output structure of a plan (library-owned, valid until the plan is released). */
const ytn_struct *ytn_plan_output(const ytn_plan_t *plan);
/* Output i of a plan with several (SVD: 0 = U, 1 = S, 2 = V); NULL past the last. */
const ytn_struct *ytn_plan_output_at(const ytn_plan_t *plan, int32_t i);
ytn_status ytn_plan_get_info(const ytn_plan_t *plan, ytn_plan_info *info);

/* The choices that a tensordot plan's first split-precision calls made with this
 * slice count (the autotuner of ytn_tensordot), and the timings behind them.
 * A choice is -1 while undecided. Timings are in ms: one run of that candidate on
 * the calling stream, the fastest of the rounds timed. A candidate that was not
 * timed reads 0, and so do all of them when a cost model decided (graph capture).
 * YTN_E_INVALID: null plan or out, or slices outside 1..6. */
typedef struct ytn_tuning {
  int32_t slices;
  int32_t auto_choice;     /* YTN_AUTO: 0 FP64, 1 split */
  int32_t split_variant;   /* 0 staged (FP64 sector matrices first), 1 fused,
                              2 fused and pipelined with the GEMM */
  int32_t tile_policy;     /* 0 128-wide tiles only, 1 with 64-wide sector tails */
  float fp64_ms, split_ms; /* YTN_AUTO: the FP64 run and the fastest split candidate */
  float staged_ms, fused_ms;
  float wide_ms, narrow_ms;
  float pipelined_ms;      /* the fused variant pipelined with the GEMM */
} ytn_tuning;
ytn_status ytn_plan_tuning(const ytn_plan_t *plan, int32_t slices, ytn_tuning *out);
void ytn_plan_release(ytn_plan_t *plan);

/* Device workspace (bytes) a ytn_tensordot call needs for this precision and
 * tolerance, or a ytn_vdot call (prec and rtol ignored); 0 for the other
 * operations. */
ytn_status ytn_workspace_size(const ytn_plan_t *plan, ytn_precision prec, double rtol,
                              size_t *bytes);

/* Workspace (bytes) with which a ytn_tensordot call stages page-locked host
 * operands on the device: ytn_workspace_size plus device copies of A, B and C.
 * Given at least this much, a call whose a, b or c is host memory moves them
 * with the copy engines (cudaMemcpyAsync on its stream, no SM time, so that a
 * call on another stream keeps every SM) instead of reading and writing host
 * memory from the data-mover kernels. Tensordot plans only (YTN_E_INVALID). */
ytn_status ytn_workspace_size_staged(const ytn_plan_t *plan, ytn_precision prec, double rtol,
                                     size_t *bytes);

/* C = tensordot(A, B) (Sec. II.B contraction equation): gather the blocks of A
 * and B into one matrix per charge sector, multiply the sectors in one grouped
 * launch, scatter the products into the blocks of C. Complex operands
 * (YTN_COMPLEX128) are contracted as real sector matrices with doubled rows
 * (A: real parts, then imaginary) or columns (B): one real GEMM gives the four
 * real products, which the scatter combines (re = re.re - im.im, im = re.im +
 * im.re); C is complex when either operand is. a, b, c: buffers of
 * sizes a->size, b->size and ytn_plan_output(plan)->size, each either device
 * memory of the context's device or page-locked host memory (cudaHostAlloc or
 * cudaHostRegister, mapped into the device's address space). Host-resident
 * data is read (and C written) by the data-mover kernels directly over the
 * host link, with no staging copy. Pageable host memory is rejected
 * (YTN_E_INVALID). Every element of c is written. prec/rtol select the product precision (rtol is the target
 * relative Frobenius error of the split path, ignored for FP64).
 * workspace: device buffer of at least ytn_workspace_size bytes, 256-byte
 * aligned. res (optional, host): filled before return. Asynchronous on stream.
 * YTN_AUTO (no counterpart in the paper) picks, per plan and slice count, the
 * faster of the FP64 path and the split path when the split path meets rtol:
 * the first such call times both paths on the caller's stream (it runs both,
 * leaves the split result in c and synchronises the stream); later calls reuse
 * the cached choice. While the stream is being captured into a graph, a cost
 * model of the two kernels' tile-padded work decides instead. res->precision
 * reports the path that wrote c; the workspace is ytn_workspace_size(YTN_AUTO).
 * The split path has two variants for plans whose blocks have at most three
 * dims per side (ytn_plan_info.split_fused): slices built straight from the
 * blocks (fused), or from FP64 sector matrices gathered first (staged). The
 * first split-precision call on such a plan (explicit or through YTN_AUTO) times
 * both on the caller's stream in the same way (three times each when a round of
 * candidates takes under 20 ms, keeping each one's fastest) and caches the
 * faster; under graph capture the fused one is taken when the blocks are large
 * (an average of at least 1024 elements per block part). Operands read straight
 * from page-locked host memory (no staging workspace) always take the staged
 * variant, whose gathers read every block linearly over the host link.
 * A large plan (sectors enough for at least two groups of about an eighth of the
 * useful FLOPs and two waves of 128-wide tiles each) also times the fused variant
 * pipelined with the GEMM: the sectors in groups, each group's slices built on
 * the lowest-priority stream of the context while the previous group's GEMM runs
 * on its highest-priority stream (a slicing CTA shares each SM with a GEMM CTA),
 * forked from and joined to the caller's stream; one pipelined call is enqueued
 * at a time per context, and a call on a stream being captured into a graph does
 * not pipeline. res->split_variant reports the variant used.
 * Likewise the split GEMM's tile list: 128 x 128 tiles, or the same with a
 * 128 x 64 last column tile for every sector whose N ends in the first half of a
 * 128-wide tile (half of that tile's padded products saved); the first split call
 * times both when the plan has such sectors (all 128 wide under graph capture);
 * res->narrow_tiles reports the choice.
 * On the split path the call also checks its own accuracy on the device (see
 * ytn_error_report): sectors whose data-aware estimate exceeds rtol are
 * recomputed on the FP64 path before C is written, and when even that leaves
 * the estimate above rtol the next ytn_sync on the context returns
 * YTN_E_TOLERANCE. The slice count comes from an a-priori forecast for typical
 * data (s = 5 at rtol 1e-10, s = 6 down to about 1.5e-11); the device check makes
 * every result meet rtol whatever its data.
 * Errors: YTN_E_INVALID (wrong plan kind), YTN_E_WORKSPACE, YTN_E_TOLERANCE
 * (rtol below what the split path can reach), YTN_E_CUDA (launch). */
ytn_status ytn_tensordot(ytn_plan_t *plan, const double *a, const double *b, double *c,
                         ytn_precision prec, double rtol, void *workspace,
                         size_t workspace_bytes, ytn_result *res, ytn_stream stream);

/* The accuracy record (ytn_error_report) of the last split-precision
 * ytn_tensordot of `plan` that ran with `workspace` (the record lives in the
 * workspace, so the next call that uses it overwrites it). Waits for `stream`,
 * then copies the record to *out. Errors: YTN_E_INVALID (null argument, not a
 * tensordot plan, or no split-precision call has completed in this workspace),
 * YTN_E_CUDA. No counterpart in the paper. */
ytn_status ytn_tensordot_report(const ytn_plan_t *plan, const void *workspace, ytn_error_report *out,
                                ytn_stream stream);

/* C = tensordot(A, B) on the FP64 path without a caller workspace and without
 * allocating anything. The paper has no counterpart: this is for callers that
 * cannot allocate device memory, for instance code inside a host application
 * that reserves all device memory for its own pool, or code that must not call
 * cudaMalloc for its latency and implicit synchronisation. The plan must exist
 * already (ytn_plan uploads its tables once). The workspace is a static 64 MiB
 * array inside the library, present on every GPU that loads the library until
 * the process exits; plans whose FP64 workspace (ytn_workspace_size) exceeds
 * 64 MiB are rejected with YTN_E_WORKSPACE. The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress, with that device current);
 * make that first call before any stream capture. Every call uses the same
 * array: calls that overlap on the GPU (other streams, other threads) race and
 * must be serialised by the caller. a, b, c may be device memory or page-locked
 * host memory, as for ytn_tensordot; host operands are staged through the rest of
 * the array when they fit beside the workspace, else read over the host link.
 * Results are those of ytn_tensordot with YTN_FP64. Errors: as ytn_tensordot
 * (YTN_E_INVALID for a plan that is not a tensordot plan or belongs to a
 * host-only context), plus YTN_E_WORKSPACE (too large) and YTN_E_UNSUPPORTED
 * (device index 64 or above). */
ytn_status ytn_tensordot_noalloc(ytn_plan_t *plan, const double *a, const double *b, double *c,
                                 ytn_stream stream);

/* out = fuse(a) / unfuse(a) (Sec. II.B). a: buffer of the planned input's
 * size; out: buffer of ytn_plan_output(plan)->size elements, every element
 * written (fused entries with no stored block are zero). Buffers may be device
 * memory or page-locked host memory, as for ytn_tensordot.
 * Asynchronous on stream. Errors: YTN_E_INVALID (wrong plan kind), YTN_E_CUDA. */
ytn_status ytn_fuse(ytn_plan_t *plan, const double *a, double *out, ytn_stream stream);
ytn_status ytn_unfuse(ytn_plan_t *plan, const double *a, double *out, ytn_stream stream);

/* out = trace of a over the planned leg pairs. Same buffer rules as ytn_fuse. */
ytn_status ytn_trace(ytn_plan_t *plan, const double *a, double *out, ytn_stream stream);

/* out = <A, B>, the sum over the elements of the blocks present in both
 * tensors of conj(A's element) times B's, in FP64 (a VDOT plan; ||A||^2 =
 * <A, A>). The paper leaves norms, overlaps and expectation values to its
 * backend; they are FP64 reductions here. a, b: buffers of the planned sizes;
 * out: one double (real tensors) or two, real and imaginary part (complex
 * tensors; both operands must have the same element type); each device memory
 * or page-locked host memory, as for ytn_tensordot. workspace: device buffer of
 * ytn_workspace_size bytes (8 bytes, 16 for complex, per CTA share of 8192
 * doubles), 256-byte aligned. Deterministic: the same call gives the same bits.
 * Asynchronous on stream. Errors: YTN_E_INVALID (wrong plan kind, null buffer),
 * YTN_E_WORKSPACE, YTN_E_CUDA. Planning errors (YTN_E_SIGNATURE,
 * YTN_E_DIM_MISMATCH, YTN_E_FUSION_MISMATCH, YTN_E_INVALID, YTN_E_UNSUPPORTED
 * for a real and a complex tensor) come from ytn_plan. */
ytn_status ytn_vdot(ytn_plan_t *plan, const double *a, const double *b, double *out, void *workspace,
                    size_t workspace_bytes, ytn_stream stream);

/* out = swap_gate(a) (a SWAP_GATE plan): every block of a copied to the same
 * place in out, negated when both groups of legs have odd parity (Sec. IV).
 * out may be a itself (in place). a, out: buffers of the plan's size, device
 * memory or page-locked host memory as for ytn_tensordot. Bit-exact.
 * Asynchronous on stream. Errors: YTN_E_INVALID (wrong plan kind, null
 * buffer), YTN_E_CUDA. */
ytn_status ytn_swap_gate(ytn_plan_t *plan, const double *a, double *out, ytn_stream stream);

/* Block-diagonal SVD (an SVD plan): every sector matrix of a is gathered into the
 * workspace and factored by the dense solver of the CUDA toolkit (SVD by polar
 * decomposition, one call per sector on stream, which waits for the host part of
 * each call; the paper leaves this to the backend), then U, S and V are written
 * to u, s, v (buffers of their planned sizes; device or page-locked host memory). Singular vectors are unique up to sign (and rotation
 * within repeated values). workspace: ytn_workspace_size bytes (the sector
 * matrices, the factors, the solver's buffer). The first SVD plan of a context
 * creates the solver handle. Errors: YTN_E_INVALID, YTN_E_WORKSPACE, YTN_E_CUDA
 * (a solver error included). */
ytn_status ytn_svd(ytn_plan_t *plan, const double *a, double *u, double *s, double *v, void *workspace,
                   size_t workspace_bytes, ytn_stream stream);

/* Block-diagonal Hermitian eigendecomposition (an EIGH plan): as ytn_svd, with
 * the toolkit's divide-and-conquer eigensolver per sector and outputs U and S. */
ytn_status ytn_eigh(ytn_plan_t *plan, const double *a, double *u, double *s, void *workspace,
                    size_t workspace_bytes, ytn_stream stream);

/* out = slice of a (a SLICE plan). Bit-exact copies. Asynchronous on stream. */
ytn_status ytn_slice(ytn_plan_t *plan, const double *a, double *out, ytn_stream stream);

/* out = conj(a) (a CONJ plan): each block copied to its place with the
 * imaginary parts of complex elements negated (real data copied as it is).
 * out may be a itself. Buffers as for ytn_swap_gate. Bit-exact. Asynchronous on
 * stream. Errors: YTN_E_INVALID (wrong plan kind, null buffer), YTN_E_CUDA. */
ytn_status ytn_conj(ytn_plan_t *plan, const double *a, double *out, ytn_stream stream);

/* Number of CTAs (one per SM) of the persistent split-precision GEMM of this
 * context; 0 (the default) uses every SM. Leaving some SMs free lets the data
 * movers of another call, for instance one that reads its operands from host
 * memory over the host link, run beside a contraction's GEMM instead of after
 * it. No counterpart in the paper. Errors: YTN_E_INVALID (host-only context, or
 * nsms outside [0, number of SMs]). */
ytn_status ytn_ctx_set_gemm_sms(ytn_ctx *ctx, int nsms);

/* Networks (Sec. II.B: general networks are contracted through pairwise
 * tensordot by the einsum / ncon convenience functions; labels in the ncon
 * convention of Pfeifer, Evenbly, Singh and Vidal, 2015).
 * tensors[i]: the structure of tensor i; labels: concatenated, tensors[i]->rank
 * per tensor. A positive label is summed and appears on exactly two legs; the
 * negative labels -1, -2, ... name the output legs in that order. Evaluation
 * order: while positive labels remain, take the smallest; a label twice on one
 * tensor traces every label that tensor carries twice; else the two tensors that
 * carry it are contracted over every label they share (tensordot(first in list
 * order, second), shared labels ascending), the result taking the first one's
 * place; what is left is joined by outer products in list order; last, the
 * legs are permuted into -1, -2, .... Each call has its own cached plan (made
 * now); the network object holds them. Errors: YTN_E_INVALID (labels), the
 * planning errors of the calls, YTN_E_UNSUPPORTED (a network of one rank-0
 * tensor). Release with ytn_ncon_release. */
ytn_status ytn_ncon_plan(ytn_ctx *ctx, int32_t ntensors, const ytn_struct *const *tensors,
                         const int32_t *labels, ytn_ncon_t **out);
/* The same network from einsum subscripts (Sec. II.B: einsum and ncon differ
 * only by syntax), e.g. "abc,cd->adb": one letter per leg; a letter on two legs
 * is summed (twice on one tensor: a trace), a letter on one leg is an output leg,
 * in the order after "->" (alphabetical without it). Summed letters become ncon
 * labels 1, 2, ... in the order of their first appearance. Errors: YTN_E_INVALID
 * (subscripts), then as ytn_ncon_plan. */
ytn_status ytn_einsum_plan(ytn_ctx *ctx, const char *subscripts, int32_t ntensors,
                           const ytn_struct *const *tensors, ytn_ncon_t **out);
/* Output structure (library-owned, valid until the network is released). */
const ytn_struct *ytn_ncon_output(const ytn_ncon_t *nc);
/* Useful FLOPs of all contractions and the number of library calls. */
ytn_status ytn_ncon_info(const ytn_ncon_t *nc, double *useful_flops, int32_t *ncalls);
/* Workspace bytes of ytn_ncon: every intermediate (256-byte aligned), then one
 * contraction workspace shared by the calls (the largest ytn_workspace_size). */
ytn_status ytn_ncon_workspace_size(const ytn_ncon_t *nc, ytn_precision prec, double rtol, size_t *bytes);
/* Run the network: data[i] is tensor i's buffer, out the output's (device or
 * page-locked host memory, as for ytn_tensordot; intermediates stay in the
 * device workspace). Every contraction uses prec / rtol. Asynchronous on stream.
 * Errors: YTN_E_WORKSPACE and those of the calls. */
ytn_status ytn_ncon(ytn_ncon_t *nc, const double *const *data, double *out, ytn_precision prec, double rtol,
                    void *workspace, size_t workspace_bytes, ytn_stream stream);
void ytn_ncon_release(ytn_ncon_t *nc);

/* Self-test of the failure path (no counterpart in the paper): enqueue on stream
 * a kernel that waits, bounded to about 2 ms, for a flag that nothing sets, then
 * records a code in the context's status word, as every bounded device wait of
 * the library does when it runs out. The next ytn_sync returns YTN_E_TIMEOUT
 * (and clears the word); the context stays usable. Nothing faults or hangs.
 * Errors: YTN_E_INVALID (host-only context), YTN_E_CUDA (launch). */
ytn_status ytn_selftest_timeout(ytn_ctx *ctx, ytn_stream stream);

/* Wait for the stream (at most timeout_ms; < 0 waits without limit) and report
 * the context's device status word: YTN_E_TIMEOUT if a bounded device wait
 * ran out since the last call, else YTN_E_TOLERANCE if a split-precision
 * contraction's result is estimated above its rtol even after the FP64
 * recomputation (the word is then cleared), YTN_E_CUDA if the stream reported
 * an error. */
ytn_status ytn_sync(ytn_ctx *ctx, ytn_stream stream, int64_t timeout_ms);

/* ---------------------------------------------------------------------------
 * Graphs: batching a sequence of calls (for instance the contractions and
 * fusions of one corner-transfer-matrix step, Sec. III Fig. 3) into one CUDA
 * graph that the host launches with a single call. No counterpart in the paper.
 * Between ytn_graph_begin and ytn_graph_end, execution calls on `stream` (a
 * created stream, not the default stream) are recorded instead of run; the
 * data and workspace buffers they name stay owned by the caller, must stay
 * valid while the graph exists, and are reused by every launch. The graph
 * holds a reference to each plan that a recorded call used (released by
 * ytn_graph_destroy), so the caller may release its own. One capture per
 * context at a time (YTN_E_INVALID otherwise); a CUDA failure in capture or
 * instantiation returns YTN_E_CUDA and leaves no graph. Phase timing is not
 * recorded while a stream is being captured.
 * ------------------------------------------------------------------------- */
typedef struct ytn_graph_s ytn_graph_t;
ytn_status ytn_graph_begin(ytn_ctx *ctx, ytn_stream stream);
ytn_status ytn_graph_end(ytn_ctx *ctx, ytn_stream stream, ytn_graph_t **graph);
ytn_status ytn_graph_launch(ytn_graph_t *graph, ytn_stream stream);
void ytn_graph_destroy(ytn_graph_t *graph);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of contraction requests (no counterpart in the
 * paper, whose CTM drivers run one contraction at a time).
 *
 * A server owns `nslots` CUDA streams and an admission thread. Submitted
 * requests wait in FIFO order; a request is admitted as soon as a slot is free
 * and its workspace (ytn_workspace_size for its precision) fits in the device
 * arena the caller handed over (the HBM budget for workspaces; inputs and
 * outputs stay wherever the caller keeps them). Admitted requests run
 * concurrently on their slots' streams, overlapping on the device; a finished
 * request releases its slot and its arena range. Each request computes exactly
 * what ytn_tensordot computes alone (no cross-request state), so its result does
 * not depend on what else runs. Times are milliseconds on the server's steady
 * clock (ytn_server_now_ms).
 * ------------------------------------------------------------------------- */
typedef struct ytn_server_s ytn_server_t;

typedef struct {
  int64_t id;          /* the caller's request id                               */
  int32_t status;      /* ytn_status of the request                             */
  int32_t slot;        /* stream slot it ran on                                 */
  double t_arrive;     /* arrival time given at submission                      */
  double t_admit;      /* admitted (slot and arena range granted, launched)     */
  double t_done;       /* completion observed by the server                     */
  size_t workspace;    /* arena bytes it held                                   */
} ytn_request_info;

/* arena: device buffer of arena_bytes (256-byte aligned) owned by the caller for
 * the server's lifetime. Errors: YTN_E_INVALID, YTN_E_CUDA. */
ytn_status ytn_server_create(ytn_ctx *ctx, int nslots, void *arena, size_t arena_bytes,
                             ytn_server_t **server);

/* Queue C = tensordot(A, B) for `plan` (a, b, c: device buffers as for
 * ytn_tensordot). t_arrive < 0 means now. Requests larger than the whole arena
 * fail at once with YTN_E_WORKSPACE (reported through ytn_server_poll). */
ytn_status ytn_server_submit(ytn_server_t *server, int64_t id, ytn_plan_t *plan, const double *a,
                             const double *b, double *c, ytn_precision prec, double rtol,
                             double t_arrive);

/* Move up to `max` finished requests into out[]; *n receives the count. */
ytn_status ytn_server_poll(ytn_server_t *server, ytn_request_info *out, int64_t max, int64_t *n);

/* Wait until every submitted request has finished (at most timeout_ms; < 0
 * without limit). YTN_E_TIMEOUT if some are still running. */
ytn_status ytn_server_drain(ytn_server_t *server, int64_t timeout_ms);

/* Current time on the server's clock, in milliseconds. */
double ytn_server_now_ms(const ytn_server_t *server);

/* Drains, stops the admission thread and destroys the streams. */
void ytn_server_destroy(ytn_server_t *server);

/* Phase timing. While enabled on a context, every execution call on its plans
 * records a CUDA event pair on the call's stream around each kernel phase
 * (events come from a pool created by ytn_profile_enable; when the pool is
 * used up, further phases are counted in `dropped` and not timed).
 * ytn_profile_read waits for the recorded events, adds their durations per
 * phase into *out and clears the record. Phases: */
enum {
  YTN_PHASE_GATHER_A = 0,   /* blocks of A -> sector matrices                 */
  YTN_PHASE_GATHER_B = 1,   /* blocks of B -> sector matrices                 */
  YTN_PHASE_GEMM = 2,       /* grouped GEMM (FP64 or split-precision)         */
  YTN_PHASE_SCATTER = 3,    /* sector matrices -> blocks of C                 */
  YTN_PHASE_SPLIT = 4,      /* FP64 -> BF16 slices (split path)               */
  YTN_PHASE_MOVE = 5,       /* fuse / unfuse / trace                          */
  YTN_PHASE_REDUCE = 6,     /* scalar products                                */
  YTN_PHASE_CHECK = 7,      /* split path: accuracy check and FP64 fallback   */
  YTN_NPHASES = 8
};
typedef struct {
  int64_t calls[YTN_NPHASES];
  double ms[YTN_NPHASES];
  int64_t dropped;
} ytn_profile;
ytn_status ytn_profile_enable(ytn_ctx *ctx, int enable);
ytn_status ytn_profile_read(ytn_ctx *ctx, ytn_profile *out);

/* Message of the last failed call on this thread (empty if none). */
const char *ytn_last_error(void);

/* Library version string. */
const char *ytn_version(void);

#ifdef __cplusplus
}
#endif

#endif /* YTN_H */
