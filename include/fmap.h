/*
 * fmap.h — C ABI of the GB300 functional-map hot path.
 *
 * Operation (DeepShapeMatchingKit, arXiv 2604.10377, Sec. 3.1):
 *   Eq. 1      A = Phi_X^+ F_X, B = Phi_Y^+ F_Y, with Phi^+ = Phi^T diag(M) for an
 *              M-orthonormal Laplace-Beltrami basis Phi (n x k), lumped mass M (n)
 *              and per-vertex features F (n x d).
 *   Eq. 2-3    C minimises ||C A - B||^2 + lambda * sum_ij D_ij C_ij^2 with
 *              D_ij = (Lambda_Y(i) - Lambda_X(j))^2 (or a caller-given mask D).
 *   Eq. 4-7    row i of C solves (A A^T + lambda diag(D_i)) c_i = (B A^T)_i.
 *   Eq. 8-9    all rows of all pairs are solved as one batch.
 * The backward pass (adjoint of Eq. 5 and chain rule of Eq. 1) is not in the
 * paper; it is given at fmap_solve_backward.
 *
 * Conventions for every call:
 *  - Every matrix is row-major. Every pointer named "device" is CUDA device
 *    memory on the context's device; the caller owns it and keeps it alive and
 *    unchanged in place while any call that reads it may still be running.
 *  - Calls only enqueue work on `stream` (a cudaStream_t passed as void*; NULL is
 *    the legacy default stream) and never synchronise or allocate device memory;
 *    scratch comes from the caller's workspace. They may therefore be captured
 *    into a CUDA graph. Calls on one batch must not overlap in time.
 *  - Return value: FMAP_OK, or an argument / launch error detected on the host
 *    (nothing was enqueued in that case). Numerical failures are reported per
 *    pair, asynchronously, in the device array `status` (see fmap_status).
 *  - Nothing crosses the boundary as an exception.
 */
#ifndef FMAP_H_
#define FMAP_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define FMAP_API __attribute__((visibility("default")))
#else
#define FMAP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes and per-pair status codes. A per-pair status word is 0 (OK) or
 * code | (row << 8), where row is the row system that failed (for NOT_SPD). */
enum fmap_status {
    FMAP_OK = 0,
    FMAP_ERR_INVALID_ARG = 1,   /* null pointer, bad index, size mismatch */
    FMAP_ERR_UNSUPPORTED = 2,   /* k > 304, d % 16 != 0, misaligned ld, ... */
    FMAP_ERR_CUDA = 3,          /* a CUDA runtime call failed (see fmap_last_cuda_error) */
    FMAP_ERR_NOT_SPD = 4,       /* per pair: a row system had a non-positive pivot */
    FMAP_ERR_NONFINITE = 5,     /* per pair: NaN/Inf in the result */
    FMAP_ERR_TIMEOUT = 6,       /* per pair: a bounded device-side wait gave up */
    FMAP_ERR_WORKSPACE = 7      /* workspace pointer NULL, too small or misaligned */
};

/* Feature precision of a batch. */
enum fmap_precision {
    FMAP_PREC_FP32 = 0,  /* F is FP32; projection error ~1e-6 relative */
    FMAP_PREC_BF16 = 1   /* F is BF16 (its values are exact inputs); FP32 accumulation */
};

typedef struct fmap_options {
    int32_t precision;          /* enum fmap_precision */
    int32_t ir_steps;           /* iterative-refinement steps after the FP32 Cholesky solve (0..3, default 1) */
    int32_t hi_gram_min_k;      /* pairs with k >= this accumulate A A^T in FP64 (default 200) */
    int32_t store_factors_max_k;/* fmap_solve saves Cholesky factors for pairs with k <= this when a
                                   `saved` buffer is given; larger pairs are refactored in the
                                   backward pass (default 304: store everything) */
    int32_t adjoint_ir_steps;   /* refinement steps of the adjoint row solves (0..3, default 0: the
                                   FP32 factor solve alone is far inside the gradient tolerance) */
    /* Tuning knobs (0 = the built-in choice). They change how work is cut into tiles and
     * launches, never the arithmetic of an output element beyond the order of its
     * partial sums; the autotuner (paper_2604_10377_gb300.autotune) searches them. */
    int32_t proj_max_stages;    /* tensor-core projection: pipeline depth cap, 2..6 (default 6) */
    int32_t proj_seg_max_v;     /* tensor-core projection of BF16 features: longest vertex segment
                                   accumulated in TMEM before a partial is written, multiple of
                                   64 in 2048..16384 (default 8192); FP32 features always use
                                   512 (accuracy of the three TF32 passes) */
    int32_t bwd_group_features; /* tensor-core backward projection: features per CTA group,
                                   64 or 128 (default 128) */
    int32_t bwd_chunk_v;        /* tensor-core backward projection: largest vertex chunk of a work
                                   item, multiple of 128 in 1024..65536 (default 8192) */
    int32_t solve_threads_k64;  /* row-solve block for k <= 64: 64 or 128 threads (default 64) */
    int32_t solve_threads_k128; /* row-solve block for 64 < k <= 128: 128 or 256 (default 128) */
    /* Persistent CTAs of the tensor-core projections, 1..152 (0 = one per SM, 152). A batch
     * whose projection runs beside another batch's row solves (two streams) can keep it on
     * part of the SMs, so that the solves' blocks hold the rest. */
    int32_t proj_ctas;          /* forward projection */
    int32_t bwd_ctas;           /* backward projection, even (two CTAs share each vertex tile) */
    int32_t solve_no_g_copy;    /* row solves of k <= 128: 0 keeps a copy of G in shared memory for the
                                   refinement residual (default), 1 reads G from L2 instead (less shared
                                   memory per block, more blocks per SM) */
    int32_t adjoint_kernel;     /* W = Gamma^T C + C^T Gamma, dA_x = Gamma^T A_y - W A_x, dA_y = Gamma A_x,
                                   and the training loss's E = C C^T - I, dL/dC = 4 E C + 2 (C - C_gt):
                                   1 tensor cores (three TF32 passes), 2 CUDA cores (FP32 FMA tiles);
                                   0 the built-in choice: tensor cores when dA_x has at least two
                                   128-column tiles per SM, else CUDA cores */
    int32_t adjoint_features;   /* tensor-core adjoint GEMMs: output columns per CTA, 64, 128 or 256
                                   (default 128, or 64 below two dA_x tiles per SM) */
    int32_t adjoint_stages;     /* tensor-core adjoint GEMMs: shared-memory stages per CTA, 1 or 2
                                   (default 1) */
} fmap_options;

typedef struct fmap_shape_desc {
    int64_t n;             /* vertices, >= 1 */
    int32_t k;             /* basis size, 1..304 */
    int32_t d;             /* feature dimension, multiple of 16, <= 4096 */
    const float* phi;      /* device, n x ld_phi FP32, columns 0..k-1 used (M-orthonormal basis) */
    int64_t ld_phi;        /* >= k, multiple of 4 (16-byte rows) */
    const float* mass;     /* device, n FP32: the diagonal of M */
    const float* evals;    /* device, k FP32 eigenvalues, or NULL if every pair using the
                              shape passes an explicit mask */
    const void* feat;      /* device, n x ld_feat, FP32 or BF16 per the batch precision */
    int64_t ld_feat;       /* >= d, multiple of 8 */
    void* dfeat;           /* device, same layout and type as feat: receives dL/dF in
                              fmap_solve_backward; NULL = do not compute it */
    float* dfeat_f32;      /* BF16 batches only (ignored in FP32 batches): device, n x ld_feat
                              FP32, 16-byte aligned, or NULL. When given together with dfeat,
                              fmap_solve_backward also writes dL/dF here in FP32, the values
                              before their rounding to BF16 (a copy for checking the backward
                              projection without the BF16 storage error) */
} fmap_shape_desc;

typedef struct fmap_pair_desc {
    int32_t shape_x;       /* source shape (basis of the columns of C) */
    int32_t shape_y;       /* target shape (basis of the rows of C); d_x == d_y. The basis
                              sizes may differ: C is k_y x k_x, with k_y row systems of
                              size k_x (the paper's pairs have k_x == k_y) */
    float lambda;          /* regularisation weight, >= 0 */
    const float* mask;     /* device k_y x k_x FP32 mask D (row i = target basis index), or
                              NULL: D_ij = (evals_y[i] - evals_x[j])^2 */
    const float* lambda_rows;  /* device, k_y FP32 weights >= 0, or NULL: row i of C then solves
                              (G + lambda_rows[i] diag(D_i)) c_i = R_i in place of lambda (the
                              regulariser sum_i lambda_i sum_j D_ij C_ij^2); read by the row solves
                              of fmap_solve and fmap_solve_backward, not checked for sign */
    float* d_lambda_rows;  /* device, k_y FP32, or NULL: with lambda_rows, fmap_solve_backward writes
                              dL/dlambda_i = -sum_j D_ij Gamma_ij C_ij here */
} fmap_pair_desc;

/* Sizes of a batch's buffers. Offsets: A of shape s starts at float a_offset(s) of
 * the flat A buffer (k_s x d_s, row-major); C of pair p at float c_offset(p) of the
 * flat C buffer (k_y x k_x of the pair, row-major). Offsets are prefix sums in input
 * order. */
typedef struct fmap_sizes {
    int64_t a_floats;        /* length of the flat A buffer (also dA) */
    int64_t c_floats;        /* length of the flat C buffer (also dC, mask gradients) */
    int64_t ws_bytes;        /* workspace for fmap_project and fmap_solve */
    int64_t ws_bwd_bytes;    /* workspace for fmap_solve_backward (and everything else) */
    int64_t saved_bytes;     /* factor storage for pairs with k <= store_factors_max_k */
    int32_t n_shapes;
    int32_t n_pairs;
} fmap_sizes;

typedef struct fmap_ctx fmap_ctx;
typedef struct fmap_batch fmap_batch;

/* Library version string (static storage). */
FMAP_API const char* fmap_version(void);

/* Human-readable text of a return or status code (static storage). */
FMAP_API const char* fmap_error_string(int32_t code);

/* Text of the last CUDA error seen by this thread's calls (static thread-local storage). */
FMAP_API const char* fmap_last_cuda_error(void);

/* Fill *opt with the defaults: FP32, ir_steps 1, hi_gram_min_k 200, store_factors_max_k 304,
 * adjoint_ir_steps 0, every tuning knob 0 (built-in choice). */
FMAP_API int32_t fmap_default_options(fmap_options* opt);

/* Create a context on CUDA device `device` (host only; no device memory is touched
 * until a batch is created). opt may be NULL for the defaults. */
FMAP_API int32_t fmap_create(fmap_ctx** out, int32_t device, const fmap_options* opt);
FMAP_API int32_t fmap_destroy(fmap_ctx* ctx);

/* Host-only planning: validate shapes and pairs against `opt` and report buffer
 * sizes, without touching the GPU. Returns INVALID_ARG / UNSUPPORTED on bad input. */
FMAP_API int32_t fmap_plan_sizes(const fmap_options* opt, const fmap_shape_desc* shapes, int32_t n_shapes,
                        const fmap_pair_desc* pairs, int32_t n_pairs, fmap_sizes* out);

/* Create a batch: validates like fmap_plan_sizes, then builds the device descriptor
 * tables (the only device memory the library owns, freed by fmap_batch_destroy).
 * Every device pointer in `shapes` and `pairs` is recorded and read by later calls.
 * n_pairs == 0 is allowed (all calls are then no-ops). Host arrays are copied. */
FMAP_API int32_t fmap_batch_create(fmap_ctx* ctx, const fmap_shape_desc* shapes, int32_t n_shapes,
                          const fmap_pair_desc* pairs, int32_t n_pairs, fmap_batch** out);
FMAP_API int32_t fmap_batch_destroy(fmap_batch* batch);
FMAP_API int32_t fmap_batch_sizes(const fmap_batch* batch, fmap_sizes* out);

/* Host copies of the offsets: a_offsets[n_shapes + 1], c_offsets[n_pairs + 1] (floats). */
FMAP_API int32_t fmap_batch_offsets(const fmap_batch* batch, int64_t* a_offsets, int64_t* c_offsets);

/* Eq. 1: A_s = Phi_s^T diag(M_s) F_s for every shape s into the flat buffer a_out
 * (device, sizes.a_floats FP32). ws: device workspace of >= sizes.ws_bytes bytes,
 * 256-byte aligned. Summation order is fixed, so results are bitwise reproducible. */
FMAP_API int32_t fmap_project(fmap_batch* batch, float* a_out, void* ws, size_t ws_bytes, void* stream);

/* Eq. 4-9: for every pair p and row i, solve (A_x A_x^T + lambda diag(D_i)) c_i = (A_y A_x^T)_i
 * by Cholesky in FP32 (the Gram matrix accumulated in FP64 when k >= hi_gram_min_k),
 * followed by opt.ir_steps steps of iterative refinement, and write C_p (device flat
 * buffer, sizes.c_floats FP32).
 *   a      device flat A buffer as written by fmap_project
 *   saved  device buffer of sizes.saved_bytes for the factors, or NULL
 *   status device int32[n_pairs]: overwritten with 0 or an fmap_status | row << 8.
 *          A failed pair's C is filled with NaN. */
FMAP_API int32_t fmap_solve(fmap_batch* batch, const float* a, float* c_out, void* saved, int32_t* status,
                   void* ws, size_t ws_bytes, void* stream);

/* Adjoint of fmap_solve and fmap_project, given G = dL/dC (flat, c_offsets):
 *   gamma_i = S_i^{-1} G_i                    (S_i the row system of Eq. 5)
 *   dL/dA_y += Gamma A_x
 *   dL/dA_x += Gamma^T A_y - (Gamma^T C + C^T Gamma) A_x
 *   dL/dD    = -lambda Gamma o C              (d_mask, optional, c_offsets layout; with row
 *                                              weights row i is scaled by lambda_rows[i])
 *   dL/dlambda = -sum(D o Gamma o C)         (d_lambda[n_pairs], optional; with row weights
 *                                              the sum of the per-row gradients, which go to
 *                                              the pair's d_lambda_rows)
 *   dL/dF_s  = diag(M_s) Phi_s dL/dA_s        written to shapes[s].dfeat when non-NULL
 * Contributions of a shape used by several pairs add up (fixed order).
 *   d_c, a, c  device, as in fmap_solve (c = its output)
 *   saved      the buffer fmap_solve filled, or NULL to refactor every pair
 *   d_a        device flat buffer (a_floats) receiving dL/dA, or NULL
 *   status     device int32[n_pairs], as in fmap_solve
 *   ws         >= sizes.ws_bwd_bytes */
FMAP_API int32_t fmap_solve_backward(fmap_batch* batch, const float* d_c, const float* a, const float* c,
                            const void* saved, float* d_a, float* d_mask, float* d_lambda,
                            int32_t* status, void* ws, size_t ws_bytes, void* stream);

/* The two halves of fmap_solve_backward, for callers that put them on different streams
 * (the adjoint solves are bound by the SMs' arithmetic latency, the backward projection by
 * HBM, so one batch's projection can run beside another batch's adjoint):
 *   fmap_adjoint           everything up to dL/dA (same arguments; d_a is required), and
 *                          dL/dD, dL/dlambda; no dL/dF
 *   fmap_project_backward  dL/dF_s = diag(M_s) Phi_s dL/dA_s for every shape with a dfeat
 *                          buffer (the chain rule of Eq. 1), from d_a as fmap_adjoint wrote it
 * Both use the batch workspace (>= sizes.ws_bwd_bytes): calls on one batch must be ordered
 * (fmap_project_backward after the fmap_adjoint whose d_a it reads). Together they do
 * exactly what fmap_solve_backward does, in the same arithmetic. status (device
 * int32[n_pairs], or NULL for fmap_project_backward) is not cleared by
 * fmap_project_backward: a bounded wait that gave up sets FMAP_ERR_TIMEOUT in every pair
 * that holds no error yet, as fmap_solve_backward and fmap_adjoint do at their end. */
FMAP_API int32_t fmap_adjoint(fmap_batch* batch, const float* d_c, const float* a, const float* c,
                              const void* saved, float* d_a, float* d_mask, float* d_lambda,
                              int32_t* status, void* ws, size_t ws_bytes, void* stream);
FMAP_API int32_t fmap_project_backward(fmap_batch* batch, const float* d_a, int32_t* status, void* ws,
                                       size_t ws_bytes, void* stream);

/* The training loss of the differentiable workloads, per pair:
 *   L_p = ||C C^T - I||_F^2 + ||C - C_gt||_F^2,  dL/dC = 4 (C C^T - I) C + 2 (C - C_gt).
 * c, c_gt, d_c: device flat buffers (c_offsets); loss: device float[n_pairs]. ws as fmap_solve. */
FMAP_API int32_t fmap_loss_orth(fmap_batch* batch, const float* c, const float* c_gt, float* loss, float* d_c,
                       void* ws, size_t ws_bytes, void* stream);

/* ---- Instrumentation (no counterpart in the paper) -------------------------------
 * When timing is enabled on a batch, every kernel the library launches for it is
 * bracketed by two CUDA events recorded on the launch stream (at most 65536 launches
 * between reads). fmap_batch_read_timing synchronises on the last event, adds the
 * elapsed times per kernel kind into ms[kind] and the launch counts into launches[kind]
 * (arrays of n_kinds >= FMAP_KIND_COUNT entries, caller-owned host memory), and starts
 * a new accumulation. Enabling or disabling also starts a new accumulation. */
enum fmap_kernel_kind {
    FMAP_KIND_PROJECT = 0,        /* projection main kernel (Eq. 1) */
    FMAP_KIND_PROJECT_REDUCE = 1, /* fixed-order sum of the projection's split-K partials */
    FMAP_KIND_GRAM = 2,           /* A_x A_x^T and A_y A_x^T (Eq. 4) */
    FMAP_KIND_SOLVE = 3,          /* row-system Cholesky solve (Eq. 5-9) */
    FMAP_KIND_ADJ_SOLVE = 4,      /* adjoint row solves */
    FMAP_KIND_ADJ_GEMM = 5,       /* dA, dB, dD, dlambda from Gamma */
    FMAP_KIND_GATHER = 6,         /* per-shape sum of dA contributions */
    FMAP_KIND_PROJECT_BWD = 7,    /* dF = diag(M) Phi dA */
    FMAP_KIND_LOSS = 8,           /* training loss and dL/dC */
    FMAP_KIND_STATUS = 9,         /* status clear */
    FMAP_KIND_COUNT = 10
};
FMAP_API int32_t fmap_batch_set_timing(fmap_batch* batch, int32_t enable);
FMAP_API int32_t fmap_batch_read_timing(fmap_batch* batch, float* ms, int32_t* launches, int32_t n_kinds);

/* Peak-throughput loops, the measured denominators of the roofline fractions (no
 * counterpart in the paper). One launch of `kind` with `blocks` CTAs and `iters` rounds
 * is enqueued on `stream`; *flops_per_launch (host) receives the arithmetic it does, so
 * that flops / (CUDA-event time of the launch) is the achieved rate:
 *   FMAP_PEAK_FP32_FMA  512 threads per CTA, 8 independent FP32 FMA chains of 4 iters each:
 *                       flops = blocks * 512 * iters * 64
 *   FMAP_PEAK_FP64_FMA  the same in FP64
 *   FMAP_PEAK_TF32_MMA  one CTA per SM (pass blocks <= the SM count), tcgen05.mma
 *                       kind::tf32 M = 128, N = 256, K = 8, iters MMAs into one TMEM
 *                       accumulator: flops = blocks * iters * 524288
 *   FMAP_PEAK_BF16_MMA  the same with kind::f16 BF16 operands, K = 16:
 *                       flops = blocks * iters * 1048576
 * sink: device buffer of >= blocks 4-byte words, zeroed by the caller (the FMA loops may
 * write there; the MMA loops set word 0 to FMAP_ERR_TIMEOUT if their bounded wait gave up). */
enum fmap_peak_kind {
    FMAP_PEAK_FP32_FMA = 0,
    FMAP_PEAK_FP64_FMA = 1,
    FMAP_PEAK_TF32_MMA = 2,
    FMAP_PEAK_BF16_MMA = 3,
    FMAP_PEAK_FP32X2_FMA = 4    /* the FP32 chains of FMAP_PEAK_FP32_FMA issued two lanes at a time
                                   (packed fma.rn.f32x2): the same flops formula */
};
FMAP_API int32_t fmap_peak_loop(int32_t kind, int32_t blocks, int64_t iters, void* sink, double* flops_per_launch,
                                void* stream);

/* ---- Spatial gradient features (Sec. "Learned Scaling and Rotation in DiffusionNet") --
 * The upstream producer of the features F of a shape, fused in one kernel that writes F
 * straight into the layout fmap_shape_desc.feat describes. For every vertex v:
 *   z_v = sum_u G_vu X_u                     complex per-channel gradients, z = x + i y
 *   (Az)_re = A_re x - A_im y
 *   (Az)_im = A_re y + A_im x   (variant 0, "A": rotation and isotropic scaling)
 *           = A_re x + A_im y   (variant 1, "B": fixed +-45 degree rotations, anisotropic scaling)
 *   out[v, c] = x_c (Az)_re,c + y_c (Az)_im,c      (= Re(conj(z) o Az) for variant A)
 * with (Az)_i = sum_j A_ij z_j. The D x D complex product runs on the tensor cores
 * (tcgen05 kind::tf32: x, y truncated to TF32, A rounded to TF32, FP32 accumulation;
 * relative error ~1e-3), the gather and the final products in FP32.
 *   n           output vertices (rows of G), >= 0 (0: nothing is enqueued)
 *   row_ptr     device int64[n + 1], CSR row offsets of G into col_idx / g_vals
 *   col_idx     device int32[nnz], columns of G (vertices of X), each in [0, n_in)
 *   g_vals      device float[2 nnz]: (Re G_vu, Im G_vu) pairs, 8-byte aligned
 *   x_in        device FP32 n_in x ld_in (ld_in >= dim, multiple of 4; 16-byte aligned)
 *   dim         D: multiple of 16, 16..128
 *   a_re, a_im  device FP32 D x D row-major
 *   out         device n x ld_out, FP32 or BF16 (out_dtype = enum fmap_precision); ld_out
 *               >= dim, multiple of 8; 16-byte aligned. Columns past dim are not written.
 *   status      device int32[1]: set to 0 by the call, then FMAP_ERR_INVALID_ARG if a CSR
 *               offset or column index was out of range (that entry is skipped) or
 *               FMAP_ERR_TIMEOUT if a bounded device wait gave up
 *   ws          device workspace of >= fmap_gradient_features_ws_bytes(dim) bytes, 256-byte
 *               aligned (the tensor-core image of A, rebuilt by every call)
 * Enqueues on stream; no allocation. Calls sharing a workspace must not overlap. */
FMAP_API size_t fmap_gradient_features_ws_bytes(int32_t dim);
FMAP_API int32_t fmap_gradient_features(int64_t n, const int64_t* row_ptr, const int32_t* col_idx,
                                        const float* g_vals, int64_t nnz, int64_t n_in, const float* x_in,
                                        int64_t ld_in, int32_t dim, const float* a_re, const float* a_im,
                                        int32_t variant, void* out, int64_t ld_out, int32_t out_dtype,
                                        int32_t* status, void* ws, size_t ws_bytes, void* stream);

/* ---- Overlap-prediction metrics (Sec. "Overlap Prediction Metrics") ---------------
 * For segments s = 0 .. n_segments-1 of flat per-vertex arrays (the vertices of one
 * shape, or of one pair's predicted overlap region): a vertex is predicted overlapping
 * when scores[v] > threshold (FP32 comparison), and is truly overlapping when
 * labels[v] != 0. Counts, exact:
 *   counts[4 s + 0..3] = TP, FP, FN, TN   (device int64[4 n_segments])
 * and, when metrics is not NULL, in FP64 (device double[7 n_segments]):
 *   metrics[7 s + 0..6] = IoU TP/(TP+FP+FN), balanced accuracy (recall + specificity)/2,
 *   accuracy (TP+TN)/n, precision TP/(TP+FP), recall TP/(TP+FN), specificity
 *   TN/(TN+FP), F1 2TP/(2TP+FP+FN); a ratio whose denominator is 0 is NaN.
 *   scores       device float[seg_offsets[n_segments]] (any values; NaN never exceeds)
 *   labels       device uint8[seg_offsets[n_segments]]
 *   seg_offsets  device int64[n_segments + 1], non-decreasing, seg_offsets[0] >= 0;
 *                segment s is [seg_offsets[s], seg_offsets[s+1])
 *   max_segment_len  >= the longest segment (vertices past it are not counted)
 * n_segments <= 65535 (UNSUPPORTED above). Enqueues on stream; no allocation. */
FMAP_API int32_t fmap_overlap_metrics(const float* scores, const uint8_t* labels, const int64_t* seg_offsets,
                                      int32_t n_segments, int64_t max_segment_len, float threshold,
                                      int64_t* counts, double* metrics, void* stream);

/* ---- Allocation-free single-pair solve (no counterpart in the paper) ---------------
 * For callers that cannot allocate device memory when they solve (a memory pool they
 * do not own is frozen, a real-time thread must not enter the allocator, or a host
 * application owns all device memory): the same Gram and row-system Cholesky kernels
 * as fmap_solve for ONE pair, with every scratch byte taken from a 2 MiB array that
 * the library defines on each GPU that loads it (held until the process exits). It
 * needs no batch, no workspace, and never calls cudaMalloc or cudaFree. Square maps
 * only (both bases of size k).
 *   a_x, a_y   device, k x d FP32 row-major descriptor matrices A and B (fmap_project's
 *              output for the source and the target shape), 4-byte aligned
 *   evals_x/y  device k FP32 eigenvalues, or NULL when mask is given
 *   mask       device k x k FP32 mask D, or NULL: D_ij = (evals_y[i] - evals_x[j])^2
 *   lambda     >= 0;  ir_steps 0..3 (refinement steps, as in fmap_options)
 *   c_out      device k x k FP32 output C;  status: device int32[1] or NULL (as fmap_solve)
 *   stream     cudaStream_t passed as void*; the call only enqueues
 * The Gram matrix is accumulated in double-float when k >= 200, as in fmap_solve.
 * Returns UNSUPPORTED if k > 256 or the scratch layout of k exceeds 2 MiB.
 * The first call on a device also sets the device up (address of the scratch array,
 * kernel shared-memory limits) on the calling thread's current device; make that
 * first call before any stream capture. All calls share the one scratch array:
 * calls that overlap on the GPU race and must not be issued. */
FMAP_API int32_t fmap_solve_pair_noalloc(const float* a_x, const float* a_y, int32_t k, int32_t d,
                                         const float* evals_x, const float* evals_y, const float* mask,
                                         float lambda, int32_t ir_steps, float* c_out, int32_t* status,
                                         void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FMAP_H_ */
