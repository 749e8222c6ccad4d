/*
 * gofmm.h -- C ABI of the B300-native GOFMM library (libgofmm.so).
 *
 * GOFMM (geometry-oblivious fast multipole method, Yu, Levitt, Reiz, Biros,
 * SC'17) compresses a dense SPD matrix K, known only through its entries, into
 * a hierarchical matrix K~ = D + S + UV (§1, eq. hmatrix) and then multiplies
 * K~ by blocks of right-hand sides.  This library does the compression on the
 * host in FP64 (Alg. 2) and the evaluation U = K~ W (Alg. 7, Table 2) on one
 * GPU in hand-written sm_103a kernels.
 *
 * Conventions shared by every entry point
 *  - Return value: GOFMM_OK (0) on success, a negative GOFMM_ERR_* code
 *    otherwise; gofmm_last_error() then describes the failure (per thread).
 *  - Indices are 0-based int64.  Dense blocks are row-major.
 *  - No entry point keeps a pointer the caller passed in after it returns,
 *    except the callback context of gofmm_entries, which must stay valid for
 *    the duration of gofmm_compress / gofmm_import only.
 *  - Nothing here synchronises the device unless the entry point says so.
 */
#ifndef GOFMM_H
#define GOFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes -------------------------------------------------------- */
#define GOFMM_OK 0
#define GOFMM_ERR_ARG (-1)         /* invalid argument (null, size, mode)       */
#define GOFMM_ERR_CALLBACK (-2)    /* the entry callback returned nonzero       */
#define GOFMM_ERR_NONFINITE (-3)   /* an entry was NaN or Inf                   */
#define GOFMM_ERR_NOMEM (-4)       /* host or device allocation failed          */
#define GOFMM_ERR_CUDA (-5)        /* a CUDA runtime call failed                */
#define GOFMM_ERR_TIMEOUT (-6)     /* a bounded device wait gave up             */
#define GOFMM_ERR_UNSUPPORTED (-7) /* valid but unsupported combination         */
#define GOFMM_ERR_IO (-8)          /* file could not be read or written         */

/* ---- how entries of K are obtained (§1 problem statement) ---------------- */
#define GOFMM_GEN_CALLBACK 0 /* only through gofmm_block_fn                       */
#define GOFMM_GEN_GAUSSIAN 1 /* K_ij = exp(-|x_i-x_j|^2/(2h^2)) + shift [i==j]   */
#define GOFMM_GEN_IMQ 2      /* K_ij = 1/sqrt(1+|x_i-x_j|^2/h^2) + shift [i==j]  */

/* ---- partitioning distance (§2.1, §3) ------------------------------------ */
#define GOFMM_DIST_GRAM_L2 0      /* d_ij^2 = K_ii + K_jj - 2 K_ij ("kernel")   */
#define GOFMM_DIST_ANGLE 1        /* d_ij = 1 - K_ij^2 / (K_ii K_jj)            */
#define GOFMM_DIST_LEXICOGRAPHIC 2 /* input order (HSS-style test mode)        */
#define GOFMM_DIST_RANDOM 3       /* seeded random order                       */

/* ---- far-list construction (§2.2, Algs. 4-5) ----------------------------- */
#define GOFMM_FAR_SYMMETRIC 0 /* same-level dual traversal: K~ symmetric      */
#define GOFMM_FAR_PAPER 1     /* FindFar + MergeFar literally (cross-level)   */

/* ---- where the evaluation gets K blocks (Alg. 2 steps 10-11) ------------- */
#define GOFMM_CACHE_BLOCKS 0 /* Kba / SKba cached at compression, kept in HBM  */
#define GOFMM_CACHE_NONE 1   /* entries generated inside the evaluation kernels
                                (generator kinds only)                          */

/* ---- data types and arithmetic of gofmm_evaluate ------------------------- */
#define GOFMM_DTYPE_F64 0
#define GOFMM_DTYPE_F32 1

#define GOFMM_PREC_FP64 0   /* FP64 everywhere (parity mode; F64 data)          */
#define GOFMM_PREC_FP32 1   /* FP32 SIMT everywhere (F32 data)                  */
#define GOFMM_PREC_TF32 2   /* S2S/S2N/L2L on TF32 tensor cores, FP32 accumulate */
#define GOFMM_PREC_BF16 3   /* ... on BF16 tensor cores, FP32 accumulate        */
#define GOFMM_PREC_BF16X3 4 /* ... split BF16 (hi*hi + hi*lo + lo*hi), FP32 acc */

/* ---- tensor-core launch configuration (gofmm_set_tc_config, autotuner) --- */
#define GOFMM_SCHED_FUSED 0    /* every grouped GEMM of an evaluation in one
                                  dependency-driven persistent launch        */
#define GOFMM_SCHED_STAGED 1   /* one persistent launch per stage            */
#define GOFMM_SCHED_PAIR 2     /* one launch per stage on SM pairs: M = 256
                                  MMAs over two r-tiles (tcgen05 cta_group::2) */
#define GOFMM_SCHED_HYBRID 3   /* upward pass in one dependency-driven launch,
                                  S2S (with the S2N parent parts) one launch
                                  per level, leaves in one dependency-driven
                                  launch                                      */
#define GOFMM_ORDER_CRITICAL 0 /* fused launch: longest dependent chain first;
                                  staged launches: heaviest task first       */
#define GOFMM_ORDER_LOCAL 1    /* fused: topological, (stage, level) groups by
                                  critical path, heap order inside; staged:
                                  heap order                                 */
#define GOFMM_ORDER_SCHEDULE 2 /* fused: the order of a list schedule
                                  simulated on the host (the earliest task to
                                  be ready first, critical path among those
                                  ready); staged: heap order                 */
#define GOFMM_ORDER_READY 3    /* fused: the upward pass and S2S in the
                                  locality order, the leaves taken from a
                                  queue of tiles whose inputs are complete
                                  (a batch: the locality order); staged:
                                  heap order                                 */
#define GOFMM_ORDER_LEVELS 4   /* fused: the upward pass, then S2S level by
                                  level from the top, then the leaves;
                                  staged: heap order                         */

/*
 * Entry callback: fill out[i*nJ + j] = K(I[i], J[j]) for 0 <= i < nI,
 * 0 <= j < nJ (row-major, FP64) and return 0.  Any nonzero return aborts the
 * calling entry point with GOFMM_ERR_CALLBACK.  The library may call it with
 * any index sets and from one thread at a time.
 */
typedef int (*gofmm_block_fn)(void* ctx, const int64_t* I, int64_t nI,
                              const int64_t* J, int64_t nJ, double* out);

/* The matrix K (N x N, SPD). */
typedef struct gofmm_entries {
    int kind;             /* GOFMM_GEN_*                                       */
    int dim;              /* point dimension (generator kinds)                 */
    int64_t n;            /* N                                                 */
    const double* points; /* generator kinds: N x dim row-major host array;
                             read during the call only.  The method itself only
                             ever sees entries computed from them.             */
    double bandwidth;     /* h (Gaussian) or l (IMQ)                           */
    double diag_shift;    /* added to K_ii (generator kinds)                   */
    gofmm_block_fn fn;    /* GOFMM_GEN_CALLBACK                                */
    void* ctx;            /* passed to fn                                      */
} gofmm_entries;

/* Compression parameters (§3 "Parameter selection"). */
typedef struct gofmm_params {
    int64_t leaf_size;      /* m: leaves hold at most m indices               */
    int64_t max_rank;       /* s: skeletons hold at most s indices            */
    double tau;             /* adaptive ID tolerance (relative to |R_00|)     */
    double budget;          /* direct-evaluation budget, fraction of N/m      */
    int kappa;              /* neighbours per index                           */
    int distance;           /* GOFMM_DIST_*                                   */
    int far_mode;           /* GOFMM_FAR_*                                    */
    int cache_mode;         /* GOFMM_CACHE_*                                  */
    int n_centroid;         /* centroid sample size of Alg. 1                 */
    int n_sample;           /* sampled rows I' per ID; 0 = 2 * max_rank       */
    int ann_max_iter;       /* randomized-tree neighbour search: iterations  */
    int num_threads;        /* host threads for compression; 0 = all         */
    double ann_target_recall; /* ... stop once the sampled recall reaches it */
    int64_t knn_exact_max;  /* exhaustive neighbour search up to this N       */
    uint64_t seed;          /* seeds every random choice of the method        */
    int device;             /* CUDA device that will evaluate                 */
    int sample_device;      /* 1: generate the sampled blocks K_{I' a} of the
                               skeletonization (Alg. 2 steps 8-9) on `device`
                               in FP64, level by level; the pivoted QR and
                               the solve stay on the host (generator kinds
                               only; needs a GPU).  0: host (default)        */
} gofmm_params;

/* Figures of a compressed matrix (for the flop/byte accounting). */
typedef struct gofmm_stats_t {
    int64_t n, depth, n_leaves;
    int64_t min_rank, max_rank;     /* over non-root nodes                       */
    double mean_rank;
    int64_t near_pairs, far_pairs;  /* ordered pairs                             */
    int64_t max_near;               /* largest |Near(beta)|                      */
    /* algorithmic flops per right-hand side column (Table 2, real shapes):
       N2S and S2N count 2 s (ncols - s) per node, the T part of
       P = [I | T] Pi^T (the identity part is a copy, not arithmetic); S2S
       2 s_b s_a per far pair; L2L 2 |b| |a| per near pair */
    double flops_n2s, flops_s2s, flops_s2n, flops_l2l;
    /* entries held by the cached K blocks (near, far) */
    int64_t near_entries, far_entries;
    int64_t interp_entries;         /* sum over nodes of s * ncols               */
    int64_t skel_total;             /* sum over non-root nodes of s              */
    int ann_iterations;
    double ann_recall;
    double compress_seconds;
    int64_t interp_t_entries;       /* sum over nodes of s * (ncols - s): the T parts */
} gofmm_stats_t;

typedef struct gofmm_handle gofmm_handle;

/* Fill *p with the defaults: m 64, s 64, tau 1e-5, budget 0.03, kappa 32,
 * Gram-l2 distance, symmetric far lists, cached blocks, n_c 32, I' = 2s,
 * 10 ANN iterations / 0.8 recall, exhaustive kNN up to N = 16384, seed 0,
 * device 0. */
void gofmm_default_params(gofmm_params* p);

/*
 * Compress K (Alg. 2): neighbour search, metric tree (Alg. 1), Near (Alg. 3,
 * budget ballot, symmetrised), Far (Algs. 4-5 or the symmetric reading),
 * adaptive ID skeletons and interpolation matrices (Alg. 6, FP64 pivoted QR +
 * triangular solve) and, in GOFMM_CACHE_BLOCKS mode, the near blocks K_ba
 * and far skeleton blocks K_b~a~.  Runs on host cores only; device memory is
 * taken on the first gofmm_prepare / gofmm_evaluate.
 *   K   : entries (kind, n, points or callback).
 *   p   : parameters; NULL means gofmm_default_params.
 *   out : receives a new handle, owned by the caller (gofmm_free).
 * Errors: ERR_ARG (n < 1, leaf_size < 1, max_rank < 1, kappa < 1, tau < 0,
 * unknown mode, CACHE_NONE with a callback), ERR_CALLBACK, ERR_NONFINITE,
 * ERR_NOMEM.  On error *out is NULL and nothing is leaked.
 */
int gofmm_compress(const gofmm_entries* K, const gofmm_params* p, gofmm_handle** out);

/*
 * Upload the compressed structure to p.device and size the evaluation
 * workspace for up to r_max right-hand sides in the given precision.
 * gofmm_evaluate calls this itself when needed; call it first to keep
 * allocation out of timed regions and before capturing a stream.
 * Synchronises the device.  Errors: ERR_ARG, ERR_UNSUPPORTED, ERR_NOMEM,
 * ERR_CUDA.
 */
int gofmm_prepare(gofmm_handle* h, int64_t r_max, int precision);

/*
 * U = K~ W (Alg. 7: N2S, S2S, S2N, L2L) on the device, asynchronously on
 * `stream` (a cudaStream_t; NULL = legacy default stream).
 *   W   : device pointer, N x r row-major in the ORIGINAL index order,
 *         leading dimension ldw >= r, element type `dtype`.
 *   U   : device pointer, N x r, leading dimension ldu >= r, same dtype;
 *         overwritten (not accumulated).  W and U must not overlap.
 *   r   : number of right-hand sides, r >= 1.
 *   precision : GOFMM_PREC_*; FP64 needs DTYPE_F64, the others DTYPE_F32.
 * The handle's workspace is reused by every call: calls on one handle must
 * be ordered (same stream, or synchronised by the caller).
 * Errors: ERR_ARG, ERR_UNSUPPORTED, ERR_NOMEM, ERR_CUDA.
 */
int gofmm_evaluate(gofmm_handle* h, const void* W, int64_t ldw, void* U, int64_t ldu,
                   int64_t r, int dtype, int precision, void* stream);

/*
 * As gofmm_evaluate, but W and U are HOST pointers (pinned memory gives the
 * fastest copies).  Copies W to the device, evaluates, copies U back and
 * synchronises `stream` before returning.  With r >= 256 (and stage timing
 * off) the columns run as two chunks of whole 128-column tiles: chunk 2 is
 * copied in while chunk 1 is evaluated and chunk 1 copied out while chunk 2
 * is evaluated (two library-owned copy streams); the result is bitwise that
 * of gofmm_evaluate (columns are independent).
 */
int gofmm_evaluate_host(gofmm_handle* h, const void* W, int64_t ldw, void* U, int64_t ldu,
                        int64_t r, int dtype, int precision, void* stream);

/*
 * As gofmm_evaluate_host, but returns once the copies and the evaluation are
 * enqueued: U is final, and W may be changed, only after
 * gofmm_synchronize(h, stream) returns.  W must hold its values when the
 * call is made (its copy to the device does not wait for earlier work on
 * `stream`; the evaluation does).  Consecutive asynchronous calls on a
 * handle take three device staging slots in turn (each call waits on the
 * device until the slot's previous call has copied its U out), so the copy
 * in of one call, the evaluation of the one before and the copy out of the
 * one before that can run at once; with pinned host buffers the copies and
 * the evaluation of a stream of calls overlap.  The copies out of one
 * handle's calls run in call order, so calls writing the same U leave the
 * last call's result.  The result is bitwise that of gofmm_evaluate.
 * Errors: as gofmm_evaluate_host; a bounded wait given up is reported by
 * gofmm_synchronize.
 */
int gofmm_evaluate_host_async(gofmm_handle* h, const void* W, int64_t ldw, void* U, int64_t ldu,
                              int64_t r, int dtype, int precision, void* stream);

/*
 * As gofmm_evaluate (FP64 or FP32 precision only), but allocating nothing:
 * the evaluation's scratch lives in a fixed 32 MiB device array that the
 * library holds on every device it is loaded on until the process exits.
 * For callers that may not allocate device memory while running (a serving
 * loop with a memory budget fixed at start-up, where an allocation could
 * fail and would synchronise the device; host code under another
 * framework's allocator).  The paper has no counterpart; it is an interface
 * of this library.
 *   - The handle must already be prepared for `precision` (gofmm_prepare or
 *     an earlier gofmm_evaluate); otherwise ERR_ARG.
 *   - r in [1, 2^30] and ldw, ldu >= r, else ERR_ARG.
 *   - Needs (N + 2 * S) * r elements of scratch (S = sum of skeleton sizes,
 *     gofmm_stats skel_total), each rounded up to 256 bytes; larger calls
 *     fail with ERR_ARG and a message naming the sizes.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, device current); make it before any stream
 *     capture.
 *   - All calls share the one array: calls whose executions overlap on the
 *     GPU (different streams or handles) race on it.
 */
int gofmm_evaluate_static(gofmm_handle* h, const void* W, int64_t ldw, void* U, int64_t ldu,
                          int64_t r, int dtype, int precision, void* stream);

/*
 * Diagnostic for the bounded waits (no counterpart in the paper): the next
 * gofmm_evaluate of h in `precision` (a tensor-core precision, prepared)
 * waits on a completion count that nothing reaches.  Its kernel gives up
 * after about a second, returns, and gofmm_synchronize reports
 * GOFMM_ERR_TIMEOUT once; the handle and the CUDA context stay usable.
 */
int gofmm_debug_stall_next(gofmm_handle* h, int precision);

/*
 * Free the device copies the tensor-core precisions do not read (the
 * row-major FP64/FP32 block and interpolation stores and the CUDA-core
 * workspaces), keeping the tensor-core tiles of every precision prepared so
 * far.  A later FP64/FP32 evaluation or a new tensor-core precision rebuilds
 * what it needs.  Synchronises the device.
 */
int gofmm_trim(gofmm_handle* h);

/*
 * Wait for `stream` and report errors the kernels recorded asynchronously:
 * GOFMM_ERR_TIMEOUT when a tensor-core kernel gave up one of its bounded
 * waits (it then returned without finishing; the outputs of that call are
 * invalid; the error is reported once and cleared), GOFMM_ERR_CUDA for a
 * CUDA error.
 */
int gofmm_synchronize(gofmm_handle* h, void* stream);

/*
 * ---- Batching and serving engine ------------------------------------------
 * Many evaluations in flight at once over any mix of resident compressed
 * matrices and right-hand-side counts (the paper batches up to 8 GPU tasks
 * over streams, §2.3 CPU-GPU hybrid; here every step is one grouped launch).
 * Each evaluation advances one stage per step (gather, N2S levels, S2S, S2N
 * levels, leaf); a step packs the current stage of every admitted evaluation
 * into one persistent tensor-core launch.  Evaluations submitted between
 * steps join at the next step.  A result is bitwise identical alone or in
 * any mix (tasks never share accumulation).
 */
typedef struct gofmm_engine gofmm_engine;

/*
 * Create an engine on `device` for precision TF32, BF16 or BF16X3, with a
 * workspace pool of pool_bytes allocated now (each running evaluation takes
 * its right-hand-side workspace, (N + 2 S) * 128-column tiles in the RT
 * layout, from the pool; admission waits until it fits).  Errors: ERR_ARG,
 * ERR_UNSUPPORTED (other precisions), ERR_NOMEM, ERR_CUDA.
 */
int gofmm_engine_create(int device, int precision, int64_t pool_bytes, gofmm_engine** out);

/*
 * Queue U = K~ W for handle h (prepared for the engine's precision).  W and
 * U are device pointers (FP32, N x r, original order, ld >= r) that must stay
 * valid until the request is done.  *id receives the request id.  Nothing
 * runs until gofmm_engine_step / gofmm_engine_drain.  Errors: ERR_ARG
 * (unprepared handle, bad sizes), ERR_NOMEM (workspace larger than the pool).
 */
int gofmm_engine_submit(gofmm_engine* e, gofmm_handle* h, const void* W, int64_t ldw, void* U, int64_t ldu,
                        int64_t r, int64_t* id);

/*
 * One step on `stream`: admit queued requests whose workspace fits (FIFO),
 * then advance every admitted request by one stage.  Asynchronous; *pending
 * receives the number of requests not yet known to be finished.
 */
int gofmm_engine_step(gofmm_engine* e, void* stream, int64_t* pending);

/* *bytes = pool workspace one request of h with r right-hand sides takes. */
int gofmm_engine_workspace(const gofmm_engine* e, gofmm_handle* h, int64_t r, int64_t* bytes);

/* *state = 0 queued, 1 running, 2 done (its U is complete). */
int gofmm_engine_poll(gofmm_engine* e, int64_t id, int* state);

/* Step until every submitted request is done; synchronises `stream`. */
int gofmm_engine_drain(gofmm_engine* e, void* stream);

/* out[0..6] = steps, kernel launches, most requests in one step, completed,
 * queued, running, finishing. */
int gofmm_engine_stats(const gofmm_engine* e, int64_t* out, int n);

/* Synchronise the device and free the engine and its pool. */
int gofmm_engine_free(gofmm_engine* e);

/*
 * ---- Static batch -----------------------------------------------------------
 * A fixed list of evaluations (handle i with r[i] right-hand sides, handles
 * may repeat) planned once: workspaces allocated, the launch sequence built
 * and uploaded.  If every handle is configured for the FUSED schedule the
 * batch runs as one dependency-driven launch per 64 items (each item's
 * tiles in its own order, the items interleaved task by task); otherwise as
 * one persistent grouped launch per stage step for all items.  Either way
 * one gather per item comes first.  gofmm_batch_evaluate runs it; calls
 * with the same W/U pointers replay a CUDA graph of the whole sequence.
 */
typedef struct gofmm_batch gofmm_batch;

/* Handles must be prepared for `precision` (TF32, BF16 or BF16X3) and live on
 * one device.  Allocates the workspaces; synchronises.  Errors: ERR_ARG,
 * ERR_UNSUPPORTED, ERR_NOMEM, ERR_CUDA. */
int gofmm_batch_create(gofmm_handle* const* hs, const int64_t* r, int count, int precision, gofmm_batch** out);

/* U[i] = K~_i W[i] for every item (device FP32 pointers, original order,
 * ld >= r[i]), asynchronously on `stream`. */
int gofmm_batch_evaluate(gofmm_batch* b, const void* const* W, const int64_t* ldw, void* const* U,
                         const int64_t* ldu, void* stream);

/* out[0] = kernels the last call launched, out[1] = deferred kernel error code
 * (nonzero: a bounded wait gave up; read after synchronising). */
int gofmm_batch_info(const gofmm_batch* b, int64_t* out, int n);

int gofmm_batch_free(gofmm_batch* b);

/* Release the handle and all its host and device memory (synchronises the
 * device first).  NULL is accepted.  Fails with ERR_ARG (and frees nothing)
 * while a serving engine holds requests of the handle.  Batches made from
 * the handle must be freed first. */
int gofmm_free(gofmm_handle* h);

/*
 * Write the compressed structure (tree order, Near/Far lists, skeletons,
 * interpolation matrices, parameters) to `path` as a flat little-endian
 * binary file (checkpoint).  Cached K blocks are not written.
 */
int gofmm_export(const gofmm_handle* h, const char* path);

/*
 * Read a structure written by gofmm_export.  K supplies entries for the
 * cached blocks (CACHE_BLOCKS) or the in-kernel generator (CACHE_NONE); it
 * must describe the same matrix as at export time.
 */
int gofmm_import(const char* path, const gofmm_entries* K, int cache_mode, int device,
                 gofmm_handle** out);

/* Figures of the compressed matrix. */
int gofmm_stats(const gofmm_handle* h, gofmm_stats_t* s);

/*
 * Stage timing.  enable = 1: gofmm_evaluate runs one launch per stage and
 * records CUDA events on its stream around each stage (a diagnostic
 * breakdown).  enable = 2: the production path with events: under the
 * fused schedule of the tensor-core precisions (the default) every grouped
 * GEMM is one dependency-driven launch, whose time is reported as stage 1
 * with stages 2-4 reading zero; under the staged schedule (and on the CUDA
 * cores) the stages are timed one by one.  enable = 0: off (repeated calls may replay a CUDA
 * graph).  gofmm_stage_times then synchronises on the last
 * event and fills ms[0..5] with the milliseconds of the last call's stages
 * (0 gather of W into tree order, 1 N2S upward pass, 2 S2S (on the CUDA
 * cores one launch; on the tensor cores one launch per level, top-down, each
 * node's task also taking its parent's S2N part), 3 S2N pushes level by level
 * (CUDA cores; zero on the tensor cores), 4 leaf S2N+L2L with scatter,
 * 5 whole call)
 * and, if n > 6, ms[6] with the number of kernels the call launched.
 */
int gofmm_set_timing(gofmm_handle* h, int enable);
int gofmm_stage_times(gofmm_handle* h, float* ms, int n);

/*
 * Structure views (for tests and tools).  Each copies into caller memory
 * and returns the element count; pass out = NULL to query the count.
 *   what = 0: perm (tree position -> original index), N int64
 *   what = 1: leaf offsets, n_leaves + 1 int64
 *   what = 2: near lists as CSR: n_leaves + 1 offsets, then the leaf numbers
 *   what = 3: far lists as CSR over heap ids: n_nodes + 1 offsets, then heap ids
 *   what = 4: skeletons as CSR over heap ids (root empty)
 *   what = 5: interpolation matrices P of all nodes in heap order, each
 *             s x ncols row-major (ncols = leaf size for a leaf, s_l + s_r
 *             otherwise), concatenated as doubles
 * A negative return is an error code (unknown `what`, NULL handle).
 */
int64_t gofmm_view(const gofmm_handle* h, int what, void* out);

/*
 * Tensor-core launch configuration of one tensor-core precision (TF32, BF16,
 * BF16X3) of a handle.  The paper has no counterpart (its GPU tasks were
 * grouped by hand, §2.3); it is an interface of this library.  Every
 * configuration computes bitwise the same U: a task's summation order does
 * not depend on how tasks are cut or ordered.
 *   piece    : 128 or 256, the tallest task piece (the MMA N ceiling); taller
 *              blocks are cut into pieces.  128 halves the block part of a
 *              shared-memory stage (4 stages of 48 KB instead of 3 of 64 KB)
 *              at the cost of reading each right-hand-side tile once per
 *              piece; blocks of at most piece / 2 rows feed two r-tiles from
 *              one TMEM buffer.
 *   schedule : GOFMM_SCHED_*.
 *   order    : GOFMM_ORDER_* (tile order inside the launches).
 * A new `piece` rebuilds the precision's plan if one exists (synchronises
 * the device); batches made from the handle before that refuse to run
 * (ERR_ARG), and the call fails with ERR_ARG while a serving engine holds
 * requests of the handle.  Default: 256, FUSED, CRITICAL.  Errors: ERR_ARG.
 */
int gofmm_set_tc_config(gofmm_handle* h, int precision, int piece, int schedule, int order);
int gofmm_get_tc_config(const gofmm_handle* h, int precision, int* piece, int* schedule, int* order);

typedef struct {
    int piece, schedule, order; /* the configuration chosen and applied        */
    int from_cache;             /* 1: taken from the cache file, none measured */
    int n_candidates;           /* candidates measured by this call            */
    int cand_piece[16], cand_schedule[16], cand_order[16];
    float cand_ms[16];          /* median ms of one evaluation (one batch call) */
    char key[32];               /* signature: structure(s), r, precision, GPU  */
} gofmm_tune_t;

/*
 * Autotuner.  Times gofmm_evaluate of h with r right-hand sides in a
 * tensor-core precision under each candidate configuration (piece 256 and
 * 128, each with the FUSED and HYBRID schedules in CRITICAL, LOCAL and
 * SCHEDULE order and the STAGED and PAIR schedules in LOCAL order: 16
 * candidates, 14 without cached blocks (no PAIR); 3 warm-up and 7 timed
 * calls each, CUDA events on `stream`, on a scratch W of pseudo-random
 * values and a scratch U the library allocates), applies the fastest with
 * gofmm_set_tc_config and reports all of them in *out.
 * cache_path (may be NULL): a JSON file of earlier choices.  If it holds
 * an entry for the same key (the structure's signature, ceil(r/128),
 * precision, GPU name and SM count), that choice is applied without
 * measuring (from_cache = 1; this needs no GPU); otherwise the new choice
 * is added to the file (written to a temporary file, then renamed).
 * A file that is not such a cache is an error and is left alone.
 * Errors: ERR_ARG (bad precision or r, unreadable/unwritable cache),
 * ERR_CUDA, ERR_NOMEM, ERR_TIMEOUT.
 */
int gofmm_autotune(gofmm_handle* h, int64_t r, int precision, const char* cache_path, void* stream,
                   gofmm_tune_t* out);

/*
 * The same for a static batch (gofmm_batch_create): the candidates are
 * piece 256 and 128, each with the FUSED schedule (the batch runs as one
 * dependency-driven launch per 64 items) and the STAGED one (one grouped
 * launch per stage step), in LOCAL order, applied to every handle; each is
 * timed as a whole batch call.  Create the batch after tuning.
 */
int gofmm_autotune_batch(gofmm_handle* const* hs, const int64_t* r, int count, int precision,
                         const char* cache_path, void* stream, gofmm_tune_t* out);

/* The cache key gofmm_autotune (count = 1) or gofmm_autotune_batch would
 * use, written to key (32 bytes, NUL-terminated).  Needs no GPU. */
int gofmm_autotune_key(gofmm_handle* const* hs, const int64_t* r, int count, int precision, char* key);

/* Description of the last error on this thread ("" if none). */
const char* gofmm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GOFMM_H */
