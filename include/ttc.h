/*
 * ttc.h -- C ABI of libttc: GB300-native tensor permute-scale-add.
 *
 * The operation (Springer, Sankaran, Bientinesi, "TTC: A Tensor Transposition
 * Compiler for Multiple Architectures", arXiv 1607.01249, section 1, Eq. 1):
 *
 *     B[Pi(i0,...,iN-1)] <- alpha * A[i0,...,iN-1] + beta * B[Pi(i0,...,iN-1)]
 *
 * Conventions (all fixed by the paper unless marked "reading"):
 *  - Layout: column-major (section 1, footnote 2): index 0 has stride 1 and
 *    indices are stored left to right.
 *  - Permutation: perm[d] is the index of A that becomes index d of B
 *    (section 2.1, Fig. 2b/2c: perm=2,1,0 on A(i0,i1,i2) gives B(i2,i1,i0);
 *    Fig. 3: perm=0,2,1 on A(m1,m2,k) gives B(m1,k,m2)).  B's size along d is
 *    sizes[perm[d]].
 *  - Outer sizes ("multiple leading dimensions", section 2.1, Table 1
 *    --lda/--ldb, Fig. 2): each index of A (and of B) may live in a larger
 *    extent, so A and/or B can be sub-tensors of larger tensors.  The stride of
 *    index k is the product of the outer sizes of indices 0..k-1.  NULL means
 *    the tensor is dense (outer = sizes).  outer_sizes_B is given in B's own
 *    index order (reading: the paper does not say).
 *  - Precision (reading): the compute type is FP64 when A or B is FP64, else
 *    FP32.  alpha and beta are rounded once to it.  FP32 compute evaluates
 *    r = fmaf(beta, b, fl32(alpha*a)), FP64 compute r = fma(beta, b,
 *    fl64(alpha*a)); r is rounded once (round-to-nearest-even) to B's type.
 *    beta == 0: B is not read.  alpha == 1 and beta == 0 with equal types: a
 *    bit copy.  Mixed types follow the paper's mixed-precision transpositions
 *    (section 2.1, --dataType=sd/ds).
 *  - FP8 E4M3 output (OCP E4M3, max 448, saturating): code =
 *    RNE_satfinite(fl32(fl32(alpha*a) / scale)); scale is either supplied by
 *    the caller (ttc_plan_set_fp8_scale) or computed on the device as
 *    fl32(amax/448), amax = max |fl32(alpha*a)| over the sub-tensor (NaN
 *    ignored; scale = 1 if amax is 0, infinite, or amax/448 underflows).  Only
 *    beta == 0 is supported with FP8 output.
 *  - Complex types (section 2.1 --dataType=c,z,cz,zc; reading for the
 *    arithmetic, which the paper does not spell out): alpha and beta are
 *    complex (ttc_plan_complex; ttc_plan gives them zero imaginary parts).
 *    The compute type is double-complex when A or B is double-complex, else
 *    single-complex; each part of alpha and beta is rounded once to it.  With
 *    alpha = (ar, ai), beta = (br, bi), a = (x, y), b = (u, v), each element
 *    evaluates, in this order,
 *        re = fl(ar*x), im = fl(ar*y);
 *        if ai != 0: re = fma(-ai, y, re), im = fma(ai, x, im);
 *        if beta != 0: re = fma(br, u, re), im = fma(br, v, im);
 *                      if bi != 0: re = fma(-bi, v, re), im = fma(bi, u, im);
 *    and rounds each part once (round-to-nearest-even) to B's type.  With real
 *    scalars each part is therefore updated exactly as a real tensor of the
 *    part's type would be.  alpha = 1, beta = 0 with equal types is a bit copy.
 *
 * Streams: every call that takes a ttc_stream_t enqueues work on that CUDA
 * stream (a cudaStream_t; NULL = the legacy default stream) and returns
 * without synchronising, unless stated otherwise.  Pointers named d_* or
 * A/B in execute calls are device pointers on the current device.
 *
 * Errors: every call returns a ttc_status; nothing aborts.  ttc_last_error()
 * gives a human-readable detail for the calling thread's last failure.
 */
#ifndef TTC_H_
#define TTC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t (same underlying type), named here so that this header does
 * not need the CUDA headers. */
typedef struct CUstream_st* ttc_stream_t;

typedef enum {
    TTC_F32 = 0,       /* IEEE binary32 ("s" in the paper's --dataType) */
    TTC_F64 = 1,       /* IEEE binary64 ("d") */
    TTC_BF16 = 2,      /* bfloat16 (output of a fused downcast, or input) */
    TTC_FP8_E4M3 = 3,  /* OCP FP8 E4M3 (output only, with a per-tensor scale) */
    TTC_C64 = 4,       /* single-complex ("c"): (real, imaginary) binary32 pair, 8 bytes */
    TTC_C128 = 5       /* double-complex ("z"): (real, imaginary) binary64 pair, 16 bytes */
} ttc_dtype;

typedef enum {
    TTC_OK = 0,
    TTC_ERR_INVALID_PERM = 1,      /* perm is not a permutation of 0..ndim-1, or ndim out of range */
    TTC_ERR_INVALID_SIZE = 2,      /* a size is negative, or the problem is too large */
    TTC_ERR_INVALID_OUTER = 3,     /* an outer size is smaller than its size */
    TTC_ERR_UNSUPPORTED_DTYPE = 4, /* dtype pair (or FP8 with beta != 0) not supported */
    TTC_ERR_ALIAS = 5,             /* the byte ranges of A and B overlap (Eq. 1 is out of place) */
    TTC_ERR_ALIGN = 6,             /* a pointer is not aligned to its element size */
    TTC_ERR_OOM = 7,               /* host or device allocation failed */
    TTC_ERR_CUDA = 8,              /* a CUDA runtime call failed (see ttc_last_error) */
    TTC_ERR_TIMEOUT = 9,           /* a bounded wait gave up */
    TTC_ERR_BUDGET = 10,           /* a request exceeds the server's memory budget */
    TTC_ERR_INVALID_ARG = 11,      /* NULL handle/pointer or bad argument */
    TTC_ERR_NOT_READY = 12         /* polled work has not finished yet */
} ttc_status;

#define TTC_MAX_DIM 16

typedef struct ttc_plan_s* ttc_plan_t;

/*
 * ttc_plan -- describe one permute-scale-add (Eq. 1; section 2.1 Table 1:
 * --perm, --size, --dataType, --beta, --lda, --ldb) and prepare it: validate,
 * drop size-1 indices, merge neighbouring indices into super-indices where
 * the memory layout allows it (section 2.1 stage 1, footnote 5), and choose a
 * kernel schedule (tile extents, vector widths, order of the flat grid).
 *
 *  out            receives the plan handle (owned by the caller; free with
 *                 ttc_plan_destroy).
 *  ndim           1..TTC_MAX_DIM.
 *  perm[ndim]     B index d is A index perm[d].
 *  sizes[ndim]    extents of A's indices (>= 0; any 0 makes the plan a no-op).
 *  outer_sizes_A  NULL or ndim outer extents of A (in A's index order).
 *  outer_sizes_B  NULL or ndim outer extents of B (in B's index order).
 *  dtype_in/out   types of A and B.  Supported pairs: f32->{f32,f64,bf16,e4m3},
 *                 f64->{f64,f32}, bf16->{bf16,f32,e4m3}, c64->{c64,c128},
 *                 c128->{c128,c64}.
 *  alpha, beta    the scalars of Eq. 1 (rounded once to the compute type;
 *                 real: for complex types their imaginary parts are 0).
 *
 * Host-only: no CUDA call is made; device resources are created on the first
 * execution on each device.  Thread-safe.
 */
ttc_status ttc_plan(ttc_plan_t* out, int ndim, const int* perm, const int64_t* sizes,
                    const int64_t* outer_sizes_A, const int64_t* outer_sizes_B,
                    ttc_dtype dtype_in, ttc_dtype dtype_out, double alpha, double beta);

/*
 * ttc_plan_complex -- ttc_plan with complex scalars alpha = alpha_re + i
 * alpha_im and beta = beta_re + i beta_im (evaluated as in the conventions
 * above).  Nonzero imaginary parts need complex tensors
 * (TTC_ERR_UNSUPPORTED_DTYPE otherwise); any part not finite gives
 * TTC_ERR_INVALID_ARG.  beta != 0 means either part is nonzero.
 */
ttc_status ttc_plan_complex(ttc_plan_t* out, int ndim, const int* perm, const int64_t* sizes,
                            const int64_t* outer_sizes_A, const int64_t* outer_sizes_B,
                            ttc_dtype dtype_in, ttc_dtype dtype_out, double alpha_re, double alpha_im,
                            double beta_re, double beta_im);

/*
 * ttc_execute -- run the plan: B <- alpha*A + beta*B under the permutation
 * (Eq. 1), asynchronously on `stream`.
 *  A   device pointer to element (0,...,0) of A (of its sub-tensor when outer
 *      sizes are given); must be aligned to the size of dtype_in.
 *  B   device pointer to element (0,...,0) of B; aligned to dtype_out.  Only
 *      elements of the sub-tensor are read or written.
 * Returns TTC_ERR_ALIAS if the byte ranges spanned by A and B overlap.  The
 * caller owns A, B and the stream; A and B must stay valid until the work on
 * `stream` has completed.  A size-0 plan returns TTC_OK without launching.
 * Launch errors are reported as TTC_ERR_CUDA.  Concurrent executions of one
 * plan on different streams are allowed except for FP8 plans that compute
 * their scale (they share the plan's amax scratch word).
 */
ttc_status ttc_execute(ttc_plan_t plan, const void* A, void* B, ttc_stream_t stream);

/* Release the plan and its device resources (waits for nothing: the caller
 * must not destroy a plan while work that uses it is still queued). */
ttc_status ttc_plan_destroy(ttc_plan_t plan);

/*
 * FP8 scale control (fused downcast; the per-tensor scale is this library's
 * addition to the paper's mixed-precision transpositions).
 *  ttc_plan_set_fp8_scale: d_scale = device pointer to one float read by
 *    every later execution (the caller keeps it alive), or NULL to compute the
 *    scale from amax on each execution (the default).
 *  ttc_plan_get_fp8_scale: enqueue on `stream` a copy of the scale used by the
 *    plan's most recent execution into d_scale_out (device pointer to one
 *    float).  Only valid after an execution on the current device.
 */
ttc_status ttc_plan_set_fp8_scale(ttc_plan_t plan, const float* d_scale);
ttc_status ttc_plan_get_fp8_scale(ttc_plan_t plan, float* d_scale_out, ttc_stream_t stream);

/* What the planner made of the problem (for tests and tooling). */
typedef enum {
    TTC_VARIANT_EMPTY = 0,    /* nothing to do */
    TTC_VARIANT_COPY = 1,     /* perm keeps index 0: long runs streamed directly */
    TTC_VARIANT_TILE = 2,     /* tile staged in shared memory between A's and B's runs */
    TTC_VARIANT_ROWCOPY = 3,  /* perm keeps index 0 with short runs: multi-row blocks, no staging */
    TTC_VARIANT_TMA_TILE = 4  /* two indices swapped: tiles copied into shared memory by the TMA */
} ttc_variant;

typedef struct {
    int ndim;                      /* canonical number of indices after dropping/merging */
    int perm[TTC_MAX_DIM];         /* canonical permutation */
    int64_t sizes[TTC_MAX_DIM];    /* canonical sizes (A order) */
    int64_t stride_A[TTC_MAX_DIM]; /* element strides of the canonical indices in A */
    int64_t stride_B[TTC_MAX_DIM]; /* element strides of the canonical indices in B (A order) */
    int64_t n;                     /* number of elements transposed */
    int64_t algorithmic_bytes;     /* n*(sA+sB) for beta == 0, n*(sA+2sB) otherwise */
    int variant;                   /* ttc_variant */
    int tile_c, tile_a, tile_b;    /* tile extents: common inner run, A-side run, B-side run */
    int64_t ntiles;                /* tiles (or rows for the copy variant) of one execution */
    int vec_in, vec_out;           /* vector widths (elements) the schedule uses when aligned */
    int candidate;                 /* index of the schedule in the plan's candidate list */
    int ncandidates;               /* number of candidate schedules the planner kept */
    int lanes_a, lanes_b;          /* tile variant: lanes along the A run / B run of the warp-mapped
                                      kernel (32, 64, 128), or 0 for the generic tile kernel */
    int slot_tables;               /* generic tile kernel: whole tiles read their per-thread
                                      offsets from precomputed slot tables (1) or walk the
                                      indices (0) */
    int packed_threads;            /* tile variant: threads per CTA (256 or 512) of the
                                      packed-lane kernel, whose lane groups run over the
                                      tile's rows without idling at run ends; 0 otherwise */
    int packed_rows;               /* tile variant with a common inner run (perm keeps
                                      index 0): positions per thread and row of the
                                      packed-row kernel, which copies the tile's rows
                                      directly without staging; 0 otherwise */
} ttc_plan_info;

ttc_status ttc_plan_get_info(ttc_plan_t plan, ttc_plan_info* info);

/*
 * Autotuner (replaces the paper's candidate search of section 2.1 stages 2-6
 * and 2.2-2.3): time up to max_candidates of the plan's candidate schedules
 * (tile extents, vector widths, order of the flat grid) on the current device
 * and keep the fastest.  Timing uses temporary device buffers that the call
 * allocates and frees itself (the caller's tensors are not touched), on
 * `stream`; the call synchronises that stream.  The choice is remembered in a
 * process-wide cache keyed by the canonical problem and device, so later plans
 * of the same problem start from it.  best_ms (may be NULL) receives the
 * winning time per execution in milliseconds.
 */
ttc_status ttc_plan_autotune(ttc_plan_t plan, int max_candidates, ttc_stream_t stream,
                             float* best_ms);

/* Select candidate schedule `index` (0 = the planner's first choice). */
ttc_status ttc_plan_select_candidate(ttc_plan_t plan, int index);

/* Save / load the autotune cache as a text file (one line per entry). */
ttc_status ttc_tune_cache_save(const char* path);
ttc_status ttc_tune_cache_load(const char* path);

/* Human-readable name of a status, and detail of the calling thread's last
 * failure (valid until its next call into the library). */
const char* ttc_status_string(ttc_status status);
const char* ttc_last_error(void);

/* Number of CUDA kernels this library has launched in this process (all
 * threads).  Used by benchmarks to report launch counts. */
int64_t ttc_launch_count(void);

/*
 * Batches: many independent permute-scale-adds (Eq. 1) -- different
 * permutations, sizes, dtypes, alpha/beta -- launched together.  Every
 * problem is cut into tiles (the paper's macro-tiles, section 2.2); the
 * problems are grouped by class (dtype pair, beta zero or not, tile body) and
 * each class is one kernel launch with one CTA per tile of all its problems,
 * each tile processed with its own problem's parameters (a per-tile record
 * names the problem).  This is the scheduling of the macro-tiles of section
 * 2.2 across thread blocks, extended across problems.
 *
 *  ttc_batch_create   new empty batch (host only).
 *  ttc_batch_add      append (plan, A, B): the plan must stay alive and
 *                     unchanged while the batch is used; A and B are device
 *                     pointers as for ttc_execute (checked the same way).
 *                     FP8 plans are rejected (TTC_ERR_UNSUPPORTED_DTYPE): their
 *                     scale needs a pre-pass of its own; so are complex plans
 *                     (the batch kernels' epilogue covers the real pairs).
 *  ttc_batch_execute  enqueue the batch on `stream`: one launch per class
 *                     for the problems below the direct threshold (every
 *                     other class on a second stream of the batch, forked
 *                     from and joined back into `stream`, so that one
 *                     class's last wave overlaps the next class's first),
 *                     and beside them, on a third stream of the batch
 *                     forked and joined the same way, one single-plan
 *                     launch per problem at or above it.  The
 *                     first execution after an add builds and uploads the
 *                     descriptors and sets up the direct problems' plans
 *                     (synchronous, allocates device memory owned by the batch
 *                     and by the plans).
 *  ttc_batch_graph_launch  the same work as a CUDA graph: captured on the
 *                     first call (after the descriptors are uploaded), then
 *                     replayed with one cudaGraphLaunch per call.
 *  ttc_batch_set_direct_threshold  problems of at least min_elements
 *                     elements run as their own kernels; 0 or less (the
 *                     default) puts every problem in the batch kernels.
 *  ttc_batch_autotune  the timed search of section 2.1 stages 4-6 for the
 *                     batch body: for every distinct plan in the batch below
 *                     the direct threshold, time up to max_candidates of the
 *                     plan's batch-body schedules (tile shape, lane layout,
 *                     rows or chunks; the cost model's order, its first
 *                     choice included) as a one-problem launch of the batch
 *                     kernel on temporary tensors (the caller's are not
 *                     touched), and keep the fastest in the plan, where
 *                     every batch and server that takes the plan afterwards
 *                     finds it.  Synchronises `stream`, allocates and frees
 *                     its own device memory, and marks the batch for a
 *                     rebuild (the next execution or graph launch uploads the
 *                     new descriptors and captures a new graph).  *retuned
 *                     (may be NULL) receives how many plans changed schedule.
 *                     max_candidates < 1 returns TTC_ERR_INVALID_ARG.
 *  ttc_batch_destroy  release the batch (not the plans); no work using it may
 *                     be queued.
 *  ttc_batch_info     number of problems and of tiles of the batch.
 * Problems of one batch must not write overlapping bytes of B, and no B may
 * overlap any A of the batch (they run concurrently).
 */
typedef struct ttc_batch_s* ttc_batch_t;
ttc_status ttc_batch_create(ttc_batch_t* out);
ttc_status ttc_batch_add(ttc_batch_t batch, ttc_plan_t plan, const void* A, void* B);
ttc_status ttc_batch_execute(ttc_batch_t batch, ttc_stream_t stream);
ttc_status ttc_batch_graph_launch(ttc_batch_t batch, ttc_stream_t stream);
ttc_status ttc_batch_destroy(ttc_batch_t batch);
ttc_status ttc_batch_info(ttc_batch_t batch, int64_t* problems, int64_t* tiles);
ttc_status ttc_batch_set_direct_threshold(ttc_batch_t batch, int64_t min_elements);
ttc_status ttc_batch_autotune(ttc_batch_t batch, int max_candidates, ttc_stream_t stream, int64_t* retuned);

/*
 * Tensor contraction by Transpose-Transpose-GEMM-Transpose (TTGT; the use of
 * tensor transpositions that motivates the paper, section 1):
 *
 *     C[modes_C] <- alpha * sum over contracted labels of A[modes_A] * B[modes_B]
 *                   + beta * C[modes_C]
 *
 * Tensors are dense and column-major (index 0 stride 1).  A label (any int)
 * names an index: one in A and B but not C is contracted, one in A and C (or
 * B and C) is a free index; every label must appear in exactly two of the
 * three tensors with the same extent (labels in all three, i.e. batched
 * contractions, and labels in one tensor only are rejected with
 * TTC_ERR_INVALID_PERM).  The product is one GEMM.  With gemm_dtype TTC_BF16
 * both operands are permuted by this library's kernels into K-major BF16
 * matrices (contracted labels fastest, row pitch rounded up to 8 elements)
 * and the GEMM is this library's tensor-core kernel (tcgen05, operands
 * copied by TMA, FP32 accumulator in tensor memory).  The exact FP32 and
 * FP64 modes permute an operand into a column-major matrix unless it already
 * is one (either orientation) and run a cuBLAS GEMM in pedantic math (no
 * reduced-precision substitution).  C takes the GEMM's output directly when
 * it is laid out as [free A labels, free B labels] or the reverse, else it is
 * permuted from a workspace with the beta update of Eq. 1.
 *
 *  ttc_contraction_plan     validate and plan (host only).  dtype: type of A,
 *                           B and C; gemm_dtype: TTC_F32 (exact FP32 GEMM)
 *                           or TTC_BF16 (operands packed to bfloat16 by the
 *                           transposes, round to nearest even, products
 *                           accumulated in FP32) for dtype TTC_F32;
 *                           TTC_F64 for dtype TTC_F64.  alpha is applied by
 *                           the GEMM.  Returns TTC_ERR_INVALID_SIZE for
 *                           inconsistent extents or a GEMM extent >= 2^31.
 *  ttc_contraction_execute  enqueue on `stream` (A, B, C device pointers;
 *                           C must not overlap A or B).  Workspaces (the
 *                           permuted operands and product, an error word)
 *                           and the cuBLAS handle are created on the first
 *                           execution on a device and owned by the
 *                           contraction.
 *  ttc_contraction_check    synchronous: TTC_ERR_TIMEOUT (reported once) if
 *                           a bounded wait of the tensor-core GEMM gave up
 *                           since the last check (that execution's C is not
 *                           valid), else TTC_OK.  Sticky (reported by every
 *                           later check) if the MMAs in flight had not
 *                           finished when the kernel released its tensor
 *                           memory: tensor-core results of concurrent and
 *                           later launches on that device may be corrupt.
 *  ttc_contraction_info     GEMM extents m, n, k and which tensors are
 *                           permuted (bit 0: A, bit 1: B, bit 2: C).
 *  ttc_contraction_autotune ttc_plan_autotune (max_candidates, stream) on
 *                           each of the contraction's permute plans; in the
 *                           BF16 mode, before the first execution, it also
 *                           times the two operand permutes with the
 *                           contracted labels in B's order instead of A's
 *                           (both operands share the order) and keeps the
 *                           faster pair.  Call it before the first
 *                           execution on a device, or the permutes keep the
 *                           schedules they started with.  Synchronises
 *                           `stream`.
 *  ttc_contraction_destroy  release (no work using it may be queued).
 */
typedef struct ttc_contraction_s* ttc_contraction_t;
ttc_status ttc_contraction_plan(ttc_contraction_t* out, int nA, const int* modes_A, const int64_t* sizes_A,
                                int nB, const int* modes_B, const int64_t* sizes_B, int nC, const int* modes_C,
                                const int64_t* sizes_C, ttc_dtype dtype, ttc_dtype gemm_dtype, double alpha,
                                double beta);
ttc_status ttc_contraction_execute(ttc_contraction_t c, const void* A, const void* B, void* C,
                                   ttc_stream_t stream);
ttc_status ttc_contraction_check(ttc_contraction_t c);
ttc_status ttc_contraction_info(ttc_contraction_t c, int64_t* m, int64_t* n, int64_t* k, int* transposes);
ttc_status ttc_contraction_autotune(ttc_contraction_t c, int max_candidates, ttc_stream_t stream);
ttc_status ttc_contraction_destroy(ttc_contraction_t c);

/*
 * GEMM consuming the packing routine (the level-3 BLAS use of sub-tensor
 * transpositions, section 2.1, Figs. 2-3), on the tensor cores:
 *
 *     C = alpha * P * Bm
 *
 * P is the BF16 panel that ttc_plan(perm, sizes, outer_sizes_A, TTC_F32 ->
 * TTC_BF16, alpha 1, beta 0) would write (each element of A's sub-tensor
 * rounded to nearest even), viewed as a column-major M x K matrix: its first
 * rank_m indices form the row index m, the others the column index k.  Bm is
 * a column-major K x N BFloat16 matrix (leading dimension K), C a
 * column-major M x N FP32 matrix (leading dimension M).  P is never written
 * to memory: each CTA gathers its slice of P from A, rounds it into shared
 * memory and multiplies it on the tensor cores (tcgen05.mma, FP32
 * accumulation in tensor memory); alpha scales the FP32 accumulator.
 *
 *  ttc_packed_gemm_plan     validate and plan (host only): perm a
 *                           permutation, 1 <= rank_m < ndim, sizes >= 1,
 *                           outer >= size, A's span and M, K below 2^31,
 *                           K a multiple of 8, 1 <= n < 2^31.
 *  ttc_packed_gemm_execute  enqueue on `stream`.  A (FP32) 4-byte aligned,
 *                           B (BF16) 16-byte aligned, C 4-byte aligned; C
 *                           must not overlap A or B (TTC_ERR_ALIAS).
 *  ttc_packed_gemm_check    synchronous: TTC_ERR_TIMEOUT if a tensor-core
 *                           wait of an execution on the current device gave
 *                           up since the last check (that C is incomplete;
 *                           the error is reported once), else TTC_OK.  If
 *                           the MMAs in flight did not finish either before
 *                           the kernel released its tensor memory, the
 *                           error is sticky (reported by every later check):
 *                           tensor-core results of concurrent and later
 *                           launches on that device may be corrupt.
 *  ttc_packed_gemm_info     m, n, k.
 *  ttc_packed_gemm_set_fp8  E4M3 operands (scale_p, scale_b: device floats,
 *                           read at execution; both NULL restore BF16): P is
 *                           packed as the E4M3 codes (RNE, satfinite) of
 *                           alpha * a / *scale_p -- the codes ttc_plan with an
 *                           E4M3 output and that scale writes -- Bm is read as
 *                           E4M3 codes (K x N bytes, column-major) standing for
 *                           *scale_b * code, and C = *scale_p * *scale_b *
 *                           P Bm, FP32 accumulation (tcgen05.mma
 *                           kind::f8f6f4).  Scales must be positive and
 *                           finite.  TTC_ERR_INVALID_SIZE unless K is a
 *                           multiple of 16.
 *  ttc_packed_gemm_destroy  release (no work using it may be queued).
 */
typedef struct ttc_packed_gemm_s* ttc_packed_gemm_t;
ttc_status ttc_packed_gemm_plan(ttc_packed_gemm_t* out, int ndim, const int* perm, const int64_t* sizes,
                                const int64_t* outer_sizes_A, int rank_m, int64_t n, double alpha);
ttc_status ttc_packed_gemm_execute(ttc_packed_gemm_t g, const float* A, const void* B, float* C,
                                   ttc_stream_t stream);
ttc_status ttc_packed_gemm_check(ttc_packed_gemm_t g);
ttc_status ttc_packed_gemm_info(ttc_packed_gemm_t g, int64_t* m, int64_t* n, int64_t* k);
ttc_status ttc_packed_gemm_set_fp8(ttc_packed_gemm_t g, const float* scale_p, const float* scale_b);
ttc_status ttc_packed_gemm_destroy(ttc_packed_gemm_t g);

/*
 * Server: continuous batching of permute-scale-add requests (Eq. 1) that
 * arrive over time.  A scheduler thread admits pending requests in arrival
 * order while the bytes of admitted, unfinished requests (A's and B's
 * sub-tensor spans) stay within `budget_bytes`, groups what it admitted into
 * an epoch and launches it on a stream: consecutive requests of at most
 * `small_tiles` tiles go together into one batched launch per class (see
 * ttc_batch_*), other requests (and every FP8 or complex request) get their
 * own launch.  Epochs on different
 * streams run concurrently, so requests that arrive while others are on the
 * GPU start as soon as budget and a stream allow.  Requests fall into three
 * size classes (batchable; up to 64 MB of algorithmic bytes; larger), each
 * with `nstreams` streams of its own, the smaller classes at higher stream
 * priority, so that small requests are not held behind the thread blocks of
 * large ones.  A completion thread detects finished epochs (event queries),
 * releases their budget and stamps each request's latency (submission to
 * detected completion).
 *
 *  ttc_server_create   budget_bytes > 0; nstreams 1..16; small_tiles >= 0.
 *                      small_tiles = 0 turns batching and size classes off:
 *                      every request gets its own launch, in arrival order
 *                      over `nstreams` streams of default priority.  Uses the
 *                      current device.  Allocates its own streams, events,
 *                      pinned staging and device descriptor slots.
 *  ttc_server_submit   enqueue (plan, A, B); returns a ticket.  A and B are
 *                      device pointers owned by the caller and must stay
 *                      valid until the request completes; the plan must
 *                      outlive the request.  TTC_ERR_BUDGET if the request
 *                      alone exceeds the budget.  FP8 plans run one at a
 *                      time per plan (their amax scratch belongs to the plan).
 *  ttc_server_poll     wait up to timeout_us microseconds (0: do not wait)
 *                      for the ticket: TTC_OK when it completed,
 *                      TTC_ERR_NOT_READY if it has not, TTC_ERR_TIMEOUT if the
 *                      watchdog gave it up, another status if it failed.
 *  ttc_server_drain    wait until every submitted request has completed
 *                      (bounded by timeout_us; TTC_ERR_TIMEOUT otherwise).
 *  ttc_server_stats    counters and latency percentiles of completed requests.
 *  ttc_server_times    submission time, admission time (taken from the
 *                      queue by the scheduler), launch time (its kernel
 *                      enqueued) and detected-completion time of one request
 *                      (host steady clock, seconds); TTC_ERR_NOT_READY until
 *                      it has completed.
 *  ttc_server_destroy  drain, stop the threads, free everything.
 * The server keeps one record per submitted request (about a hundred bytes,
 * plus its latency sample) until it is destroyed: a long-running caller
 * recycles servers (their streams and slots are cheap to recreate).
 */
typedef struct ttc_server_s* ttc_server_t;

typedef struct {
    int64_t submitted, completed, failed, epochs, launches;
    int64_t bytes;                 /* algorithmic bytes of the completed requests */
    double p50_us, p90_us, p99_us, max_us, mean_us;   /* latency of completed requests */
    double first_submit_s, last_complete_s;           /* host clock, seconds */
    int64_t peak_inflight_bytes;   /* largest admitted-and-unfinished byte count seen */
} ttc_server_stats_t;

ttc_status ttc_server_create(ttc_server_t* out, int64_t budget_bytes, int nstreams, int64_t small_tiles);
ttc_status ttc_server_submit(ttc_server_t server, ttc_plan_t plan, const void* A, void* B, int64_t* ticket);
ttc_status ttc_server_poll(ttc_server_t server, int64_t ticket, int64_t timeout_us);
ttc_status ttc_server_drain(ttc_server_t server, int64_t timeout_us);
ttc_status ttc_server_stats(ttc_server_t server, ttc_server_stats_t* stats);
ttc_status ttc_server_times(ttc_server_t server, int64_t ticket, double* submit_s, double* admit_s,
                            double* launch_s, double* complete_s);
ttc_status ttc_server_destroy(ttc_server_t server);

/*
 * ttc_execute_noalloc -- ttc_execute for callers that cannot allocate device
 * memory.  The paper has no counterpart: this is a deployment aid of this
 * library.
 *
 * Who needs it: ttc_execute allocates a small per-device scratch area on a
 * plan's first execution on each device (the FP8 amax/scale words and the
 * tile schedule's offset tables).  Some callers cannot make that call: code
 * whose device memory is entirely owned by a pool allocator (a framework's
 * caching allocator, a serving process with a fixed memory budget) where a
 * cudaMalloc would fail or break the pool's accounting, and code that must
 * not make the implicitly synchronising cudaMalloc/cudaFree calls at all.
 * This entry point runs the same kernels with that scratch placed in one
 * fixed array of TTC_NOALLOC_SCRATCH_BYTES bytes that the library reserves
 * statically in device memory (every GPU that loads the library holds it
 * until the process exits).  It makes no device-memory allocation: it calls
 * no cudaMalloc, cudaMallocAsync or cudaFree and no library routine that
 * allocates device memory (host-side it only builds the kernel parameters).
 *
 *  plan, A, B, stream  as for ttc_execute (same checks, same results).
 *  d_scale_out         FP8 plans: NULL or a device pointer to one float that
 *                      receives the scale used; ignored for other plans.
 *
 * Limits and behaviour:
 *  - A plan whose schedule needs more scratch than the static array holds is
 *    rejected with TTC_ERR_INVALID_SIZE (ttc_last_error gives both sizes);
 *    ttc_execute still runs it.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture begins.  The address is looked up again when
 *    the device's CUDA context has changed since (after cudaDeviceReset, for
 *    instance), so a call never passes a kernel an address of an earlier
 *    context.
 *  - A tile schedule's offset tables are copied from host memory that the
 *    call owns only until it returns; on a stream that is being captured
 *    such a call is refused with TTC_ERR_INVALID_ARG (schedules without
 *    tables are not refused).
 *  - The schedule run is the plan's selected candidate, or, unless the caller
 *    selected one, the candidate an earlier ttc_plan_autotune remembered for
 *    this problem on this device (as ttc_execute's first use takes it).
 *  - Every call shares the one array per device, and the array keeps the last
 *    call's contents; each call re-initialises what it uses (the amax word is
 *    cleared, the offset tables are re-uploaded on `stream`).  Calls whose
 *    work overlaps on the GPU (different streams, or different host threads
 *    without ordering) race on the array and must be serialised by the
 *    caller.
 */
#define TTC_NOALLOC_SCRATCH_BYTES 8192
ttc_status ttc_execute_noalloc(ttc_plan_t plan, const void* A, void* B, float* d_scale_out,
                               ttc_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* TTC_H_ */
