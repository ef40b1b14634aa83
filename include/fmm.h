/*
 * fmm.h -- C ABI of the GB300 (sm_103a) fused Strassen GEMM library.
 *
 * Operation (Section 1, Eq. 1 and its 2x2 partitioned form, Eq. 2):
 *
 *     C = alpha * A * B + beta * C
 *
 * with A (m x k), B (k x n), C (m x n), all ROW-MAJOR with leading dimensions
 * lda >= k, ldb >= n, ldc >= n (elements, not bytes).  `levels` selects how
 * many levels of Strassen's algorithm are applied:
 *
 *   levels = 0  classical product (the library's own comparator GEMM);
 *   levels = 1  the seven products of Section 3, Eq. (3): each product
 *               M_r = (sum_q U[q,r] A_q)(sum_q V[q,r] B_q) is accumulated
 *               into every C quadrant it feeds, C_q += alpha*W[q,r]*M_r;
 *   levels = 2  the 49 two-level products (Section 3.4), i.e. the Kronecker
 *               square of the one-level table.
 *
 * Fringes (Section 3.5): each dimension d is padded with implicit zeros to
 * 2^L * h, h = roundup(ceil(d / 2^L), 8); padded rows and columns are never
 * read from or written to memory.
 *
 * Conventions shared by every entry point
 *  - Pointers A, B, C, workspace are DEVICE pointers owned by the caller; the
 *    library keeps no reference after the call returns.  `stream` is a
 *    cudaStream_t passed as void*; NULL means the legacy default stream.
 *  - Launches are asynchronous on `stream`.  A non-FMM_OK return means nothing
 *    was launched.  Faults detected on the device (a bounded wait that timed
 *    out) are reported by fmm_device_status().
 *  - beta == 0 means C is not read (BLAS convention): NaN/Inf in C vanish.
 *  - m, n or k == 0 is allowed; k == 0 only scales C by beta.
 *  - C must not overlap A, B or the workspace (FMM_ERR_ARG).
 *  - The fmm_gemm* entry points never allocate device memory; the workspace
 *    they need is sized by fmm_workspace_size*() and passed in.
 */
#ifndef FMM_GB300_H
#define FMM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum fmm_status {
    FMM_OK = 0,
    FMM_ERR_ARG = 1,          /* invalid argument (sizes, strides, aliasing) */
    FMM_ERR_ALIGN = 2,        /* alignment the selected algorithm needs is missing */
    FMM_ERR_UNSUPPORTED = 3,  /* combination not built (variant, levels, algo) */
    FMM_ERR_WORKSPACE = 4,    /* workspace missing or smaller than required */
    FMM_ERR_CUDA = 5,         /* a CUDA runtime/driver call failed */
    FMM_ERR_TIMEOUT = 6       /* a device-side bounded wait gave up */
} fmm_status;

/* Arithmetic of the sub-products.  PAPER: FP32 SIMT only (Section 2.3); the
 * tensor-core precisions below are this library's GB300 re-design. */
typedef enum fmm_variant {
    /* A, B, C float32.  Operand sums are formed in FP32, split into
     * hi = bf16(P), lo = bf16(P - hi); each product is hi*hi + hi*lo + lo*hi
     * on BF16 tensor cores with FP32 accumulation (FP32-accurate). */
    FMM_F32_SPLIT3_BF16 = 0,
    /* A, B bfloat16; C float32.  Sums formed in FP32, rounded once to BF16. */
    FMM_BF16 = 1,
    /* A, B float16; C float32.  Sums formed in FP32, scaled by a power of two
     * per (product, 128-row / column panel) so that they fit FP16, rounded once;
     * the scale is undone exactly in the epilogue. */
    FMM_F16_SCALED = 2,
    /* A, B, C float32.  Sums formed in FP32, rounded once to BF16. */
    FMM_F32_PLAIN_BF16 = 3
} fmm_variant;

/* Where the operand linear combinations are formed. */
typedef enum fmm_algo {
    FMM_ALGO_AUTO = 0,
    /* Operand sums of all 7^L products are formed by one streaming pass over
     * A and B and stored (already rounded/split) in the workspace; the
     * tensor-core kernel then loads them with TMA.  Handles any alignment. */
    FMM_ALGO_PACKED = 1,
    /* Operand sums are formed on chip while tiles are loaded (Section 3.1):
     * TMA stages the W_A (W_B) source tiles, transform warps add them with
     * their signs, round/split, and feed the tensor cores.  No workspace,
     * except for FP16 operands: the panel maxima of their operand sums, found
     * by a pass over A and B that does not store the sums.  FP32 operands in
     * both fused kernels; BF16 and FP16 operands in the tensor-memory kernel
     * (CTA pairs), forward products, FP16 with Strassen's basis.  Needs lda,
     * ldb multiples of 4 (FP32) / 8 (16-bit) and 16-byte aligned A, B. */
    FMM_ALGO_FUSED = 2,
    /* levels == 2 only: top-level sums materialised in FP32 in the workspace
     * (Section 3.4, hybrid), bottom level fused as in FMM_ALGO_FUSED. */
    FMM_ALGO_HYBRID = 3
} fmm_algo;

typedef struct fmm_options {
    int algo;       /* fmm_algo; 0 = automatic choice */
    int tile_n;     /* 0 = automatic; otherwise 128 or 256 */
    int num_ctas;   /* 0 = one persistent CTA per SM */
    int schedule;   /* order of the (product, tile) work items: 0 = automatic,
                       1 = product-major (all tiles of one product, then the next),
                       2 = tile rounds (each CTA runs all 7^L products of one output tile
                           back to back, so its destination blocks stay in L2) */
    int bk;         /* packed algorithm, split3: k-depth of a pipeline stage, 0 = automatic,
                       64 (128-byte swizzle) or 32 (64-byte swizzle, twice the stages) */
    int cta_pair;   /* packed algorithm: 0 = automatic, 1 = one CTA per 128-row tile,
                       2 = CTA pairs (clusters of two CTAs share 256-row tiles through
                           cta_group::2 UMMAs, each CTA loading half of the B tile;
                           bk must be 64) */
    int round_tiles; /* tile-rounds schedule: output tiles per round, 0 = automatic (as many
                        as keep the C blocks that one round updates within a quarter of the
                        L2 cache when C traffic dominates, else one per CTA or CTA pair) */
    int fringe;      /* sizes that do not split evenly, levels >= 1: 0 = pad (implicit zero
                        padding of every block to the padded size, Section 3.5), 1 = peel
                        (Strassen on the largest core whose sizes are multiples of 8 * 2^L,
                        then classical products for the k, row and column strips) */
    int pipeline;    /* packed algorithm, levels >= 1: 0 = automatic, 1 = off, 2 = on.  On:
                        the operand sums are formed in seven passes, one per top-level
                        product, on an internal stream, and the tensor-core kernel runs each
                        top-level product's 7^(L-1) products as soon as their sums exist, so
                        the sum passes overlap the products (joined back into `stream`).
                        The first pipelined call on a device creates that stream: make it
                        before any stream capture begins. */
    int basis;       /* 0 = Strassen (Eq. 3); 1 = the Strassen-Winograd variant written per
                        product (14 nonzeros in each of U, V, W; levels <= 1, packed or fused);
                        2 = a <3,2,3> basis of rank 15 (levels <= 1, packed or fused; A split into
                        3 x 2 blocks, B into 2 x 3, C into 3 x 3; 15 products instead of the
                        classical 18, so 5/6 of the classical MMA work against Strassen's 7/8;
                        no pipelining); 3 = the <2,3,2> basis of rank 11 (levels <= 1, packed
                        or fused; A split into 2 x 3 blocks, B into 3 x 2, C into 2 x 2:
                        Strassen's seven products on the first two block columns of A and block
                        rows of B plus the four block products of the third, 11/12 of the
                        classical MMA work; no pipelining).  Bases other than 0 form their
                        operand sums in one table-driven pass per operand. */
    int deterministic; /* 1 = ownership mode: each output tile position belongs to one CTA
                          (pair), which applies the C updates of all 7^L products in a fixed
                          order, each item's after the previous item's have completed; results
                          are bitwise reproducible (tile-rounds schedule, one tile per CTA
                          pair per round).  0 = automatic: the ownership order for one-level
                          Strassen products with beta = 0, h_k <= 512, 16-byte aligned C
                          rows and every other option at its default (there it is faster: the
                          first update of each C block stores it and the later ones find the
                          block in L2); otherwise updates from different CTAs may land in any
                          order */
    int outer_scaling; /* 1 = outside power-of-two scaling (packed, forward product): every row
                          of A and column of B is scaled by 2^-e so that its largest magnitude
                          lies in [1, 2) before the operand sums are formed, and C is scaled
                          back exactly afterwards (keeps badly scaled rows and columns from
                          losing accuracy in the Strassen sums; two more passes over C) */
    int fused_kernel; /* fused and hybrid algorithms: 0 = automatic (2 in CTA pairs, else 1);
                         1 = both operands' sums written to shared memory for the UMMAs;
                         2 = CTA pairs only: the A-operand sums stored in tensor memory
                         (tcgen05.st) and read from there by the UMMAs, the B-operand sums in
                         shared memory (half the shared-memory traffic of the operand tiles) */
    int store_first; /* packed algorithm, beta = 0, levels >= 1: 0 = automatic (on), 1 = off (C is
                        zeroed first and every product adds into it), 2 = on: the products run in
                        a few launch phases so that the first update of every C block stores it
                        (no zeroing pass, no read of C by those updates); in the deterministic
                        mode the products of each tile position run in order on one worker, so
                        the first one to update a block stores it within the single launch;
                        not with the pipelined or outside-scaling modes, nor in batched plans */
    int reserved[2]; /* zero */
} fmm_options;

/* Bytes of workspace fmm_gemm needs for this problem (0 when none).  Returns
 * (size_t)-1 for an unsupported combination. */
size_t fmm_workspace_size(int64_t m, int64_t n, int64_t k, int levels, int variant);
size_t fmm_workspace_size_ex(int64_t m, int64_t n, int64_t k, int levels, int variant,
                             const fmm_options* opt);

/* C = alpha*A*B + beta*C with `levels` Strassen levels (0, 1 or 2) in the
 * arithmetic `variant` (fmm_variant).  A and B have the element type the
 * variant names; C is float32.  `workspace` (device, >= 256-byte aligned) must
 * hold fmm_workspace_size() bytes; it may be NULL when that size is 0.
 * Classical products (levels 0): BF16 / FP16 operands whose base address and row
 * stride are 16-byte aligned are read in place (when both are, no workspace is needed and
 * `workspace` may be NULL), and with beta = 0 the product is stored into C without a
 * zeroing pass; C's old contents are never read when beta = 0, whatever the level count. */
fmm_status fmm_gemm(int64_t m, int64_t n, int64_t k, float alpha,
                    const void* A, int64_t lda, const void* B, int64_t ldb,
                    float beta, float* C, int64_t ldc, int levels, int variant,
                    void* workspace, size_t ws_bytes, void* stream);

/* As fmm_gemm, with explicit algorithm and tile options (NULL = defaults). */
fmm_status fmm_gemm_ex(int64_t m, int64_t n, int64_t k, float alpha,
                       const void* A, int64_t lda, const void* B, int64_t ldb,
                       float beta, float* C, int64_t ldc, int levels, int variant,
                       void* workspace, size_t ws_bytes, void* stream,
                       const fmm_options* opt);

/* fmm_gemm without a workspace argument, for callers that cannot allocate device
 * memory (for example a plug-in whose host application owns every device allocation,
 * or a latency-critical caller that must not call cudaMalloc / cudaFree because they
 * can synchronise the device).  The operand sums go to a scratch array built into
 * the library: 64 MiB per GPU, held from library load until process exit.  A problem
 * that needs more scratch than that is rejected with FMM_ERR_WORKSPACE; a product that
 * needs none at all (a classical product whose 16-bit operands the tensor cores read
 * in place) runs whatever fmm_workspace_size() estimates for it.  No device memory is
 * allocated.  All calls on a device share that one scratch and
 * it keeps the previous call's contents (nothing in it needs to start at zero):
 * calls whose work overlaps on the GPU race on it and must be serialised by the
 * caller.  The first call on each device looks up the scratch's device address;
 * make that first call before any stream capture begins.  Other arguments and
 * errors as fmm_gemm.  The paper has no counterpart to this entry point. */
fmm_status fmm_gemm_noalloc(int64_t m, int64_t n, int64_t k, float alpha,
                            const void* A, int64_t lda, const void* B, int64_t ldb,
                            float beta, float* C, int64_t ldc, int levels, int variant,
                            void* stream);

/* Backward of C = A * B for a differentiable linear layer: given dC = dL/dC,
 *     dA = dC * B^T   (m x k, leading dimension ldda)   and
 *     dB = A^T * dC   (k x n, leading dimension lddb),
 * each computed as a `levels`-level Strassen product (Section 3, Eq. 3) on the
 * transposed views: no transposed copy of A, B or dC is made; the operand sums
 * take the coefficients of the transposed quadrants and the tensor cores read
 * the transposed operands in their other major-ness.  A and B have the type the
 * variant names, dC is float32; dA and dB are float32 and are overwritten (either
 * may be NULL to skip it).  The two products run one after the other on `stream`
 * and share the workspace, which must hold fmm_workspace_size_backward() bytes. */
fmm_status fmm_gemm_backward(int64_t m, int64_t n, int64_t k,
                             const void* A, int64_t lda, const void* B, int64_t ldb,
                             const float* dC, int64_t lddc, float* dA, int64_t ldda,
                             float* dB, int64_t lddb, int levels, int variant,
                             void* workspace, size_t ws_bytes, void* stream);
/* As fmm_gemm_backward, with options (NULL = defaults).  The backward products run in CTA
 * pairs (cta_pair 0 or 2) on the packed algorithm (algo 0 or FMM_ALGO_PACKED), or with the
 * operand sums formed on chip (FMM_ALGO_FUSED: FP32 A and B, split3 or plain_bf16; the
 * tensor-memory kernel reads B^T and A^T as transposed tiles; no workspace); pipeline,
 * round_tiles, schedule, tile_n and num_ctas apply as in fmm_gemm_ex. */
fmm_status fmm_gemm_backward_ex(int64_t m, int64_t n, int64_t k,
                                const void* A, int64_t lda, const void* B, int64_t ldb,
                                const float* dC, int64_t lddc, float* dA, int64_t ldda,
                                float* dB, int64_t lddb, int levels, int variant,
                                void* workspace, size_t ws_bytes, void* stream,
                                const fmm_options* opt);
size_t fmm_workspace_size_backward(int64_t m, int64_t n, int64_t k, int levels, int variant);
/* Workspace of fmm_gemm_backward_ex with these options (the basis changes the block sizes);
 * (size_t)-1 for an unsupported combination. */
size_t fmm_workspace_size_backward_ex(int64_t m, int64_t n, int64_t k, int levels, int variant,
                                      const fmm_options* opt);

/* ------------------------------------------------------------------ batching
 * Many independent, unevenly sized products C_p = alpha_p A_p B_p + beta_p C_p in one
 * persistent tensor-core launch per tile width.  The paper batches instances of one
 * product by variant on blockIdx.z (Section 3.3); here every (problem, Strassen
 * product, output tile) is one item of a single work list.
 *
 * The Strassen level and tile width of each problem come from a tuning table: size
 * class i holds the problems with min(m, n, k) <= max_dim[i] (classes in increasing
 * order; larger problems fall in the last class). */
typedef struct fmm_tune_table {
    int count;            /* classes in use, 1..8 */
    int64_t max_dim[8];   /* upper bound of min(m, n, k) for class i */
    int levels[8];        /* Strassen levels for class i (0, 1 or 2) */
    int tile_n[8];        /* output tile width for class i: 128, 256 or 0 (automatic) */
} fmm_tune_table;

/* The built-in table (measured on GB300 with the split-BF16 arithmetic). */
void fmm_tune_default(fmm_tune_table* out);
/* The built-in table for a variant, which the batched entry points use when `tune` is NULL:
 * for BF16 and FP16 operands one class, classical (the classical product reads 16-bit
 * operands in place, with no pass at all); for FP32 operands fmm_tune_default's table. */
void fmm_tune_default_ex(int variant, fmm_tune_table* out);
/* Levels and tile width the table assigns to an m x n x k problem (NULL = built-in). */
fmm_status fmm_tune_select(const fmm_tune_table* tune, int64_t m, int64_t n, int64_t k,
                           int* levels, int* tile_n);

/* Native autotuner: times square d x d x d products of `variant` at levels 0, 1, 2 and
 * tile widths 128 and 256 for each probe size d = sizes[0..count-1] (1..8 sizes,
 * increasing; `reps` timed calls after one warm-up, CUDA events on `stream`), and writes
 * to *out one class per run of probes with the same fastest (levels, tile_n), class
 * boundaries at the geometric means of neighbouring probe sizes.  times_ms, if not NULL,
 * receives count * 6 times in milliseconds (probe-major, then levels, then tile 128, 256).
 * Allocates and frees its own device buffers: a tuning call, not a product call. */
fmm_status fmm_tune_measure(int variant, const int64_t* sizes, int count, int reps,
                            fmm_tune_table* out, float* times_ms, void* stream);

/* A batched plan holds, in the caller's workspace, the parameter blocks of every
 * problem (tensor maps, destination tables) and the work list.  Creating it uploads
 * them synchronously; executing it only launches kernels on `stream` (no host
 * synchronisation, no allocation, no copies), so an execution can be captured in a
 * CUDA graph and replayed while the plan, its workspace and the operands live.
 * Arrays are host arrays of length `count`; A, B, C entries are device pointers.
 * The workspace (>= 256-byte aligned) must hold fmm_batched_workspace_size() bytes. */
typedef struct fmm_batched_plan fmm_batched_plan;
size_t fmm_batched_workspace_size(int count, const int64_t* m, const int64_t* n,
                                  const int64_t* k, int variant, const fmm_tune_table* tune);
fmm_status fmm_batched_plan_create(int count, const int64_t* m, const int64_t* n,
                                   const int64_t* k, const float* alpha,
                                   const void* const* A, const int64_t* lda,
                                   const void* const* B, const int64_t* ldb,
                                   const float* beta, float* const* C, const int64_t* ldc,
                                   int variant, const fmm_tune_table* tune,
                                   void* workspace, size_t ws_bytes, fmm_batched_plan** plan);
fmm_status fmm_batched_plan_execute(const fmm_batched_plan* plan, void* stream);
void fmm_batched_plan_destroy(fmm_batched_plan* plan);
/* Plan, execute once on `stream` and release the plan. */
fmm_status fmm_gemm_batched(int count, const int64_t* m, const int64_t* n, const int64_t* k,
                            const float* alpha, const void* const* A, const int64_t* lda,
                            const void* const* B, const int64_t* ldb, const float* beta,
                            float* const* C, const int64_t* ldc, int variant,
                            const fmm_tune_table* tune, void* workspace, size_t ws_bytes,
                            void* stream);

/* Last error message of the calling host thread ("" when none). */
const char* fmm_last_error(void);

/* Synchronises `stream`, then reads and clears the device error word written
 * by bounded waits and self-checks inside the kernels.  Returns FMM_ERR_TIMEOUT
 * if any wait gave up since the previous call; FMM_ERR_CUDA on a CUDA error or a
 * failed device-side check (a CTA pair given different TMEM columns, a parameter
 * block naming a tensor map outside its table; the kernel skipped its work). */
fmm_status fmm_device_status(void* stream);

/* Limit, in nanoseconds, of every device-side wait of kernels launched after
 * this call (default 2e9).  Test hook for failure detection. */
void fmm_set_wait_timeout_ns(uint64_t ns);

/* Launches one CTA that waits on an mbarrier nothing ever arrives at, with
 * the current wait limit, then records a timeout in the device error word.
 * Exercises the bounded-wait failure path without faulting the GPU. */
fmm_status fmm_debug_wait_timeout(void* stream);

/* Writes the level-L product table (levels 0, 1 or 2) that the kernels use:
 * U[(bi * 2^L + bj) * 7^L + r] is the coefficient of block (bi, bj) of A in the
 * A-operand of product r; V likewise for B, W for the C update.  Each array
 * must hold 4^L * 7^L entries.  Returns 7^L, or -1 on a bad argument.
 * Source: Section 3, Eq. (3), and its Kronecker power for Section 3.4. */
int fmm_product_table(int levels, int8_t* U, int8_t* V, int8_t* W);
/* As fmm_product_table for a basis (fmm_options.basis: 0 Strassen, 1 Strassen-Winograd,
 * 2 the <3,2,3> basis of rank 15, 3 the <2,3,2> basis of rank 11).  With the basis's block grid (g_m, g_k, g_n) and its R
 * products (fmm_basis_shape): U[(i * g_k + l) * R + r] is the coefficient of A block (i, l)
 * in product r, V[(l * g_n + j) * R + r] that of B block (l, j), W[(i * g_n + j) * R + r]
 * that of product r in C block (i, j); U holds g_m g_k R entries, V g_k g_n R, W g_m g_n R.
 * Returns R, or -1 for a bad argument or a basis and level count that are not built. */
int fmm_product_table_ex(int levels, int basis, int8_t* U, int8_t* V, int8_t* W);

/* The store-first launch phases the library runs for beta = 0 (fmm_options.store_first):
 * phase_of[r] (R entries) receives the phase of product r, store[c * R + r] (g_m g_n R
 * entries, the layout of W above) is 1 where product r stores C block c -- the block's first
 * update -- and 0 where it adds into it or does not touch it.  Returns the number of phases,
 * or -1 (levels < 1, or a basis and level count that is not built).  Host only, no CUDA call.
 * The paper runs the instances in any order with atomic updates (Section 3.3); this planner
 * orders them so that C needs no zeroing pass. */
int fmm_store_phases(int levels, int basis, int* phase_of, int8_t* store);
/* Block grid and product count of `levels` levels of a basis: dims[0..3] = g_m, g_k, g_n,
 * R (levels 0: 1, 1, 1, 1; Strassen and Strassen-Winograd: 2^L, 2^L, 2^L, 7^L; basis 2 at
 * one level: 3, 2, 3, 15; basis 3 at one level: 2, 3, 2, 11).  Returns 0, or -1 for a
 * combination that is not built. */
int fmm_basis_shape(int levels, int basis, int* dims);

/* Phase timing.  While enabled, each launch of a phase -- 0: beta pass,
 * 1: operand-sum passes, 2: tensor-core kernel -- is bracketed by two CUDA
 * events recorded on the caller's stream.  fmm_profile_read waits for the
 * recorded events, writes the summed milliseconds and launch counts of the
 * three phases into ms[3] and launches[3] (either may be NULL) and forgets
 * them.  Measurement hook; no effect on results. */
fmm_status fmm_profile_enable(int on);
fmm_status fmm_profile_read(double* ms, int64_t* launches);

/* Library version string. */
const char* fmm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FMM_GB300_H */
