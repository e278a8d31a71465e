/*
 * bfly.h -- C ABI of the GB300 butterfly-factorization apply library (libbfly.so).
 *
 * The library applies a constructed butterfly factorization
 *
 *     K ~ U^L G^{L-1} ... G^h M^h (H^h)^* ... (H^{L-1})^* (V^L)^*          (Eq. Kfactors, Sec. 1.2)
 *
 * and its adjoint to batches of complex vectors on one GPU.  K is N x N with
 * N = n0 * 2^L; the row and column trees T_X, T_Omega are complete binary
 * trees of even depth L (Sec. 3), h = L/2 and m = 2^h.  The factors are the
 * ones produced by the construction of Sec. 3: leaf bases U^L, V^L
 * (2^L blocks of n0 x r), transfer blocks G^l, H^l (2^L blocks of r x 2r per
 * level l = h..L-1, Eq. RSh2 and Sec. 3.2.2) and the middle-level weights
 * S^h_{i,j} of M^h (Eq. KeqUMV).  The apply costs O(N log N) per vector
 * (Sec. 3.3): one pass over every factor.
 *
 * All entry points return a bf_status and never throw, abort or print.
 * Argument errors are reported before anything is launched.  Calls that take
 * a stream are asynchronous with respect to the host unless stated otherwise.
 */
#ifndef BFLY_H
#define BFLY_H

#include <stddef.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BF_OK = 0,
    BF_ERR_INVALID = 1,      /* bad argument: null pointer, odd L, aliasing in/out, ld < N, ... */
    BF_ERR_CUDA = 2,         /* a CUDA runtime call failed (the CUDA error is cleared)          */
    BF_ERR_NOMEM = 3,        /* device or host allocation failed                               */
    BF_ERR_UNSUPPORTED = 4,  /* valid but outside the library's compiled limits (r > 32, ...) */
    BF_ERR_TIMEOUT = 5,      /* a kernel's bounded wait expired; its output is not valid       */
    BF_ERR_CORRUPT = 6,      /* a factor file failed its checks (magic, sizes, checksums)      */
} bf_status;

typedef enum {
    BF_C64 = 1,              /* complex64: interleaved (re, im) float; S as float             */
    BF_C128 = 2,             /* complex128: interleaved (re, im) double; S as double          */
} bf_dtype;

/* Shape of a factorization.  Compiled limits: L even, 0 <= L <= 24;
 * 1 <= r <= 32; 1 <= leaf <= 64; and m * max(leaf, r) <= 8192 (one tree
 * node's vector segment must fit in shared memory).
 * There is no arity field: a 1D factorization (binary trees, this struct
 * with bf_plan_create) and a 2D one (quadtrees, the same struct with
 * bf_quad_create) have different factor shapes and different plans, so the
 * entry point chosen states the arity.  There is no precision field either:
 * factors are always stored in complex64 (FP32), and the operand precision
 * of the tensor-core path is a property of a plan that can change between
 * calls (bf_plan_set_precision), not of the factorization's shape. */
typedef struct {
    int L;          /* depth of T_X and T_Omega, even (Sec. 1.2)                     */
    int leaf;       /* n0 = N / 2^L, points per leaf node (Sec. 3, "bounded leaf")  */
    int r;          /* rank of every low-rank block (Sec. 3)                         */
    int nrhs_max;   /* most vectors one kernel pass processes; sizes the workspace   */
} bf_desc;

/* Host arrays of the factors in canonical layout, row-major, block index
 * first; all in the dtype given (S real).  h = L/2, m = 2^h, nb = 2^L.
 *   VL      nb blocks of n0 x r: block b is V^L_{b,0} (column leaf b).
 *   H[t]    t = 0..h-1 holds level l = h + t: nb blocks of r x 2r; block
 *           j'*2^{L-l-1} + i is H^l_{j',i} (Sec. 3.2.2).
 *   S       m*m*r reals: S[(i*m + j)*r + k] is entry k of the diagonal S^h_{i,j}
 *           (row node i, column node j; Eq. KeqUMV).
 *   G[t]    as H: block i'*2^{L-l-1} + j is G^l_{i',j} (Eq. RSh2).
 *   UL      nb blocks of n0 x r: block a is U^L_{a,0}.
 * For L = 0, H and G may be NULL. */
typedef struct {
    int dtype;                  /* bf_dtype */
    const void *VL;
    const void *const *H;
    const void *S;
    const void *const *G;
    const void *UL;
} bf_factors;

typedef struct bf_plan_s *bf_plan;

/* Builds a plan: validates the shape, packs the factors into the device
 * layouts of the forward and adjoint kernels (complex64, block-contiguous in
 * the order each thread block consumes them), uploads them, and allocates a
 * workspace of 2^L * r * nrhs_max complex64 entries.  When nrhs_max >= 8 it
 * also packs the factors for the CUDA-core multi-RHS core, and when
 * nrhs_max >= 32 (and r, n0 are multiples of 8 with blocks of at most 64 x 64)
 * for the tensor-core core -- two levels per pass multiplied out, in FP64,
 * into dense blocks -- each with its own packed streams and up to three
 * workspaces of 2^L * r * nrhs_max entries (rounded up to 128 vectors for the
 * tensor-core core): bf_plan_device_bytes reports the total.  The factor
 * arrays are copied: the caller may free them when this returns.
 * Synchronizes `stream` before returning.  On error *plan is set to NULL. */
bf_status bf_plan_create(bf_plan *plan, const bf_desc *desc, const bf_factors *factors,
                         cudaStream_t stream);

/* u = K_bf g for nrhs vectors (Eq. Kfactors applied right to left).
 *   in, out  complex64, column-major N x nrhs with leading dimension ld >= N
 *            (entries), rows in tree order (1D: natural index order).
 *            Device pointers are used in place.  Host pointers (pinned or
 *            pageable) are staged through plan-owned device buffers, which the
 *            first such call allocates; the host output is complete when
 *            `stream` completes.  On the single-vector path the copies run
 *            per group of tree nodes on plan-owned side streams forked from
 *            and joined back to `stream` (also under graph capture), so they
 *            overlap the other groups' kernels.
 *   nrhs     >= 0; 0 is a no-op.  Processed nrhs_max vectors per pass: one
 *            vector at a time through the fused single-RHS kernels (up to 4
 *            per thread block), 8..31 through the CUDA-core multi-RHS core,
 *            32 or more through the tensor-core core (bf_plan_set_precision).
 * in and out must not overlap (BF_ERR_INVALID).  The calling thread's
 * current device must be the plan's (BF_ERR_INVALID otherwise).  One plan owns one
 * workspace: calls on the same plan must not run concurrently on different
 * streams. */
bf_status bf_apply(bf_plan plan, const void *in, void *out, int nrhs, long long ld,
                   cudaStream_t stream);

/* g' = K_bf^* f = V^L H^{L-1} ... H^h (M^h)^* (G^h)^* ... (G^{L-1})^* (U^L)^* f,
 * the conjugate transpose of the factor chain (Eq. Kfactors).  Same
 * arguments and rules as bf_apply. */
bf_status bf_apply_adjoint(bf_plan plan, const void *in, void *out, int nrhs, long long ld,
                           cudaStream_t stream);

/* Releases every device and host resource of the plan (synchronizes the
 * device first).  NULL is accepted. */
bf_status bf_plan_destroy(bf_plan plan);

/* Reads and clears the plan's device error word (synchronizes `stream`):
 * BF_ERR_TIMEOUT if a kernel gave up on a bounded wait since the last check.
 * In the checked build of the library (libbfly_checked.so, compiled with
 * BF_CHECKED: the single-vector and batched kernels test every global index
 * against the extent their launch's arguments define, skip an access outside
 * it and record it): BF_ERR_INVALID if such a check fired. */
bf_status bf_plan_check(bf_plan plan, cudaStream_t stream);

/* Bytes of device memory the plan holds (factors, workspace, staging). */
size_t bf_plan_device_bytes(bf_plan plan);

/* Per-kernel timing for profiling: when enabled, every kernel the plan
 * launches is bracketed by CUDA events on the launching stream.
 * bf_plan_kernel_times synchronizes the device and returns, for the
 * "down" kernel (leaf + merging levels) and the "up" kernel (middle
 * transpose + splitting levels + leaf), the launch count and summed
 * milliseconds since the last reset, then resets them. */
bf_status bf_plan_set_profiling(bf_plan plan, int enable);
bf_status bf_plan_kernel_times(bf_plan plan, int *down_launches, double *down_ms,
                               int *up_launches, double *up_ms);

/* Apply without any device allocation: u = K_bf g (adjoint = 0) or
 * K_bf^* g (adjoint != 0) like bf_apply / bf_apply_adjoint, but the level-h
 * intermediate vector is kept in a fixed array of 2^21 complex64 entries
 * (16 MiB) compiled into the library instead of the plan's workspace, and
 * nothing is allocated, not even host-pointer staging.  The paper has no
 * counterpart: this serves callers that cannot call cudaMalloc when they
 * apply the operator -- code whose device memory is owned by another
 * allocator (a framework's caching pool that has reserved the GPU), or
 * latency-critical loops where an allocation and the device synchronization
 * it implies are not acceptable.  The plan is still created once beforehand.
 *   in, out  DEVICE pointers only (host pointers: BF_ERR_INVALID); same layout,
 *            ld and aliasing rules as bf_apply.
 *   Limit    2^L * r (one vector's level-h data) must be <= 2^21, else
 *            BF_ERR_UNSUPPORTED; larger batches run in passes of
 *            floor(2^21 / (2^L r)) vectors.
 *   Device   the calling thread's current device must be the one the plan
 *            was created on (BF_ERR_INVALID otherwise): the array is per
 *            device, the plan's factors are on one.
 * Every GPU that loads the library holds the 16 MiB array until the process
 * exits.  The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it with the
 * identity of the device's context, so after a cudaDeviceReset (which ends
 * the context; plans made before it are gone with it) the next call looks it
 * up again; make the first call on a device, and the first after a reset,
 * before any stream capture.  All calls share the one array, which
 * keeps the last call's contents (each pass overwrites what it reads, so
 * nothing needs clearing): calls that overlap on the GPU -- on different
 * streams, or from different threads -- race and give wrong results. */
bf_status bf_apply_static_scratch(bf_plan plan, const void *in, void *out, int nrhs, long long ld,
                                  int adjoint, cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * Batches of independent factorizations.  Many operators -- each its own
 * shape (L, n0, r) and its own number of vectors -- applied together: every
 * operator's down half runs in one grouped launch (one thread block per
 * operator, middle-level node and RHS tile, largest operators first), then
 * every up half in a second, optionally replayed from a CUDA graph.  Each
 * operator is the fused path of bf_apply with its own factors, packed with
 * the batch's ring configuration.  Operators with many vectors on deep trees
 * (nrhs >= route_min_rhs and L >= route_min_L) are routed instead to their
 * own CUDA-core multi-RHS passes (as bf_apply runs 8 or more vectors), which
 * read each factor once per direction instead of once per RHS tile; those
 * passes run on eight side streams beside the grouped launches (forked from
 * and joined back into the caller's stream, inside the graph too).
 * ------------------------------------------------------------------------- */
typedef struct bf_batch_s *bf_batch;

typedef struct {
    int T;              /* RHS per thread block: 1, 2, 4 or 8 (0 = 1)                  */
    int slot_kb;        /* factor ring slot size in KB (0 = 16)                         */
    int stages;         /* ring slots (0 = 2)                                           */
    int route_min_rhs;  /* route operators with at least this many vectors (0 = 8;      */
                        /* negative: route none)                                        */
    int route_min_L;    /* ... and trees at least this deep (0 = 6)                     */
} bf_batch_config;

typedef enum {
    BF_BATCH_EACH = 0,     /* one operator at a time (two launches per operator)          */
    BF_BATCH_GROUPED = 1,  /* two grouped launches for the whole batch                    */
    BF_BATCH_GRAPH = 2,    /* the grouped launches captured once in a CUDA graph, replayed */
} bf_batch_mode;

/* Builds a batch of n operators: descs[o] and factors[o] as in bf_plan_create
 * (descs[o].nrhs_max >= nrhs[o]); the vectors are bound here: in[o], out[o]
 * are DEVICE pointers to column-major N_o x nrhs[o] complex64 arrays with
 * leading dimension ld[o] (in[o] and out[o] must not overlap).  cfg may be
 * NULL.  Synchronous.  Limits as bf_plan_create; BF_ERR_UNSUPPORTED if an
 * operator's thread block does not fit the ring configuration. */
bf_status bf_batch_create(bf_batch *batch, int n, const bf_desc *descs, const bf_factors *factors,
                          const void *const *in, void *const *out, const int *nrhs, const long long *ld,
                          const bf_batch_config *cfg, cudaStream_t stream);

/* out[o] = K_o in[o] (adjoint = 0) or K_o^* in[o] for every operator of the
 * batch, by the given bf_batch_mode, asynchronously on `stream`.  The first
 * BF_BATCH_GRAPH call per direction captures and instantiates the graph
 * (on a private stream; call it before capturing anything else yourself). */
bf_status bf_batch_apply(bf_batch batch, int adjoint, int mode, cudaStream_t stream);

/* As bf_plan_check, over every operator of the batch. */
bf_status bf_batch_check(bf_batch batch, cudaStream_t stream);

/* Thread blocks per grouped launch. */
int bf_batch_items(bf_batch batch);

bf_status bf_batch_destroy(bf_batch batch);

/* ---------------------------------------------------------------------------
 * Differentiation (reverse mode).  u = K_bf g is linear in g and in each factor
 * separately, so for a real loss with upstream gradient ubar = dL/du the
 * gradients are gbar = K_bf^* ubar and, for every factor step y = A x of the
 * chain, Abar = ubar-at-y x^* summed over the vectors -- for the blocks the
 * chain uses conjugate-transposed ((V^L)^*, (H^l)^*), Bbar = x ybar^*.
 * Complex gradients follow PyTorch's convention, dL/dRe + i dL/dIm; S^h is
 * real and gets dL/dS.  These entry points work on factors held in device
 * memory in the canonical layout of bf_factors (complex64, S float), so a
 * training loop can update them in place between calls; nothing is packed.
 * ------------------------------------------------------------------------- */
typedef struct bf_diff_s *bf_diff;

/* Device arrays of the factors (inputs), complex64 and float, canonical
 * layout as in bf_factors; H and G are host arrays of h device pointers. */
typedef struct {
    const void *VL;
    const void *const *H;
    const float *S;
    const void *const *G;
    const void *UL;
} bf_dfactors;

/* Device arrays receiving the gradients, same shapes and layout as the
 * factors; written (not accumulated) by bf_diff_backward. */
typedef struct {
    void *VL;
    void *const *H;
    float *S;
    void *const *G;
    void *UL;
} bf_dgrads;

typedef struct {
    int L, leaf, r;       /* shape, as in bf_desc                                       */
    int nrhs_max;         /* most vectors per call                                      */
    int stride;           /* keep the input of every stride-th factor for the backward
                             pass (1 = every factor); 0 = choose from saved_budget       */
    size_t saved_budget;  /* with stride 0: bytes the kept inputs plus one recompute
                             segment may take (0 = keep every factor's input)            */
} bf_diff_desc;

/* Creates a differentiation plan: validates the shape (limits of bf_desc, and
 * 4 r^2 <= 4096, n0 r <= 4096), picks the checkpoint stride k and allocates
 * the plan's work buffers ((2 + k - 1) vectors of max(N, 2^L r) x nrhs_max
 * complex64).  Synchronous; *out is NULL on error. */
bf_status bf_diff_create(bf_diff *out, const bf_diff_desc *desc);
bf_status bf_diff_destroy(bf_diff plan);

/* The checkpoint stride k the plan uses: the backward pass recomputes the
 * inputs of the k - 1 factors after each kept one. */
int bf_diff_stride(bf_diff plan);

/* Bytes of the `saved` buffer bf_diff_forward fills for nrhs vectors (the
 * inputs of factors 0, k, 2k, ..., position-major complex64); 0 on bad input. */
size_t bf_diff_saved_bytes(bf_diff plan, int nrhs);

/* u = K_bf g for nrhs column-major vectors (device pointers, leading
 * dimension ld >= N, as bf_apply), keeping the checkpoints in `saved`
 * (device, bf_diff_saved_bytes(plan, nrhs) bytes, owned by the caller and
 * read by the matching bf_diff_backward).  Asynchronous on `stream`. */
bf_status bf_diff_forward(bf_diff plan, const bf_dfactors *factors, const void *g, void *u, int nrhs,
                          long long ld, void *saved, cudaStream_t stream);

/* Given ubar = dL/du (device, column-major, ld as in the forward call) and
 * the `saved` buffer of the forward call on the same factors and nrhs:
 * gbar = K_bf^* ubar and every factor's gradient into `grads`.  Recomputes
 * the inputs that were not kept.  The plan's work buffers are used:
 * calls on one plan must not run concurrently on different streams.
 * Asynchronous on `stream`. */
bf_status bf_diff_backward(bf_diff plan, const bf_dfactors *factors, const void *ubar, void *gbar, int nrhs,
                           long long ld, const void *saved, const bf_dgrads *grads, cudaStream_t stream);

/* Precision of the tensor-core multi-RHS core (batches of 32 or more RHS
 * with r, n0 multiples of 8).  Its MMAs take TF32 or BF16 operands with FP32
 * accumulation; every complex product is formed from real products.  A
 * split rung writes each FP32 value x as x_hi + x_lo, x_hi = x rounded to the
 * nearest value of the operand type, x_lo = x - x_hi (rounded again), and
 * forms a b as a_lo b_hi + a_hi b_lo + a_hi b_hi (three MMAs, small terms
 * first).  Errors are relative 2-norm errors against the FP64 apply of the
 * same factors (N = 2^16 .. 2^20, r = 16, 128 RHS).
 *   BF_PREC_FP32    (default) 3xTF32 (K = 8 per MMA): ~1e-6.
 *   BF_PREC_TF32    one TF32 product: a third of the MMAs, ~1e-3.
 *   BF_PREC_BF16X6  BF16 three-way split x = hi + mid + lo (24 mantissa bits),
 *                   six BF16 MMAs of K = 16 per product (the terms down to
 *                   2^-16): as many MMAs as 3xTF32, ~1e-6.
 *   BF_PREC_BF16X3  BF16 hi/lo split (16 mantissa bits): half the MMAs of
 *                   3xTF32, ~1e-5.
 *   BF_PREC_BF16    one BF16 product: a sixth of the MMAs of 3xTF32, ~6e-3.
 * BF16 shares FP32's exponent range, so no scaling is applied.  The fused and
 * CUDA-core paths compute in FP32 whatever is set.  BF_ERR_INVALID for any
 * other value. */
typedef enum {
    BF_PREC_FP32 = 0,
    BF_PREC_TF32 = 1,
    BF_PREC_BF16X3 = 2,
    BF_PREC_BF16 = 3,
    BF_PREC_BF16X6 = 4
} bf_precision;
bf_status bf_plan_set_precision(bf_plan plan, int precision);

/* ---------------------------------------------------------------------------
 * 2D factorizations on quadtrees.  The paper develops the factorization in
 * 1D and notes that it carries over to higher dimensions (Sec. 1.2); this is
 * that carry-over for an n x n grid, N = n^2: quadtrees of even depth L, four
 * children per node, n0 = N / 4^L points per leaf, h = L/2, m = 4^h.  Points
 * and frequencies are numbered in quadtree (Morton) order, so a node's points
 * are contiguous and child c holds its c-th quarter.  Level l uses rank
 * r_l = min(r, N / 4^l) (l = h..L).  The factors use bf_factors with these
 * shapes (row-major, block index first; nb = 4^L):
 *   VL      nb blocks of n0 x r_L: block b is V^L_{b,0}.
 *   H[t]    level l = h + t: nb blocks of r_{l+1} x 4 r_l; block
 *           j''*4^{L-l-1} + i' is H^l_{j'',i'} (column node j'' at level l+1,
 *           row node i' at level L-l-1).
 *   S       m*m*r_h reals: S[(i*m + j)*r_h + k] is entry k of S^h_{i,j}.
 *   G[t]    as H: block i''*4^{L-l-1} + j' is G^l_{i'',j'}.
 *   UL      nb blocks of n0 x r_L: block a is U^L_{a,0}.
 * The plan multiplies out, in FP64, one dense (4 r_out) x (4 r_in) block per
 * group of four vectors a level acts on (the leaf factors folded into the
 * first and last level, S^h into the first splitting level), stores them in
 * complex64 and applies them level by level on CUDA cores in FP32.
 * ------------------------------------------------------------------------- */
typedef struct bf_quad_s *bf_quad;

/* Builds a 2D plan from desc (L even, 2 <= L <= 12; leaf a power of 4 up to
 * 16; 1 <= r <= 32; nrhs_max >= 1) and host factors.  Holds both directions'
 * blocks (complex64) and two workspaces of 4^L r_h nrhs_max entries.
 * Synchronizes `stream`.  BF_ERR_INVALID for a bad shape or NULL array,
 * BF_ERR_UNSUPPORTED outside the limits, BF_ERR_NOMEM if memory runs out;
 * on error *plan is NULL. */
bf_status bf_quad_create(bf_quad *plan, const bf_desc *desc, const bf_factors *factors, cudaStream_t stream);

/* out = K_bf in (adjoint = 0) or K_bf^* in, for nrhs vectors: DEVICE
 * pointers to column-major N x nrhs complex64 arrays with leading dimension
 * ld >= N, in Morton point order; in and out must not overlap
 * (BF_ERR_INVALID, as are host pointers).  Runs in chunks of nrhs_max
 * vectors, L launches each.  Asynchronous on `stream`; calls on one plan
 * must not overlap (one workspace). */
bf_status bf_quad_apply(bf_quad plan, const void *in, void *out, int nrhs, long long ld, int adjoint,
                        cudaStream_t stream);

/* Device bytes held (blocks of both directions and workspaces), kernel
 * launches per chunk and direction (L), how many of them run on the tensor
 * cores for chunks of 32 or more vectors, and release (synchronizes the
 * device; NULL accepted). */
size_t bf_quad_device_bytes(bf_quad plan);
int bf_quad_passes(bf_quad plan);
int bf_quad_tc_passes(bf_quad plan);
bf_status bf_quad_destroy(bf_quad plan);

/* Tensor-core path of a 2D plan.  When nrhs_max >= 32 the plan also keeps
 * every level except the two that read and write the caller's vectors in
 * the tensor-core core's form (a group's stack split into output parts and
 * K-chunks of at most 64 that are multiples of 16, each a [Re F; Im F]
 * block; the K-chunks accumulate in tensor memory), and chunks of 32 or more
 * vectors run those levels on the tensor cores, with 128-vector planar tiles
 * between all levels.  bf_quad_set_precision picks the rung exactly as
 * bf_plan_set_precision does (BF16 rungs split the blocks once, synchronously);
 * bf_quad_check reads and clears the error word of the tensor-core kernel's
 * bounded waits (BF_ERR_TIMEOUT), synchronizing `stream`. */
bf_status bf_quad_set_precision(bf_quad plan, int precision);
bf_status bf_quad_check(bf_quad plan, cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * Sketch products of a 1D kernel matrix, for the construction from products
 * (Sec. 3.1, first case; the randomized SVD of Sec. 2.1 needs K_ij C_jj and
 * K_ij^* R_ii for Gaussian blocks supported on one middle-level node each).
 * The matrix is K(x_j, xi_k) = exp(2 pi i (x_j xi_k + c_j |xi_k|)) with
 * x_j = j/N, xi_k = k - N/2 (Sec. 4, Eq. 1D-FIO-kernal: Example 1 has
 * c_j = (2 + sin 2 pi x_j)/8; c = 0 is the Fourier matrix of Sec. 1.1 up to
 * the column shift).  Entries are generated on the fly (exact fixed-point
 * phase reduction modulo 1, FP32 sin/cos and sums): O(N^2 k) work, nothing
 * of K is stored.
 * ------------------------------------------------------------------------- */
typedef struct {
    int log2N;          /* N = 2^log2N, 1 <= log2N <= 30                          */
    int nb;             /* rows of one sketch block: a power of two <= N          */
    int k;              /* columns of a sketch block, 1 <= k <= 32                */
    int node0, nodes;   /* blocks used: node0 .. node0 + nodes - 1 (nodes <= 65535)*/
    long long lo, hi;   /* output index range, 0 <= lo < hi <= N                  */
    int adjoint;        /* 0: products with K; otherwise with K^*                 */
} bf_sketch_desc;

/* With b < nodes, c < k, o in [lo, hi), n = node0 + b:
 *   adjoint = 0:  out[(b k + c)(hi - lo) + o - lo] = sum_t K(o, n nb + t) blocks[(b nb + t) k + c]
 *   adjoint != 0: out[(b k + c)(hi - lo) + o - lo] = sum_t conj(K(n nb + t, o)) blocks[(b nb + t) k + c]
 * over t < nb: block b is a sketch block on column node n (forward) or row
 * node n (adjoint), and only the output rows [lo, hi) are formed.
 *   c_fixed  DEVICE array of N unsigned 64-bit integers c_j 2^64 (c_j in [0, 1)
 *            as a fixed-point fraction), or NULL for c = 0.
 *   blocks   DEVICE complex64, nodes x nb x k (row-major), caller-owned.
 *   out      DEVICE complex64, nodes x k x (hi - lo), caller-owned, must not
 *            overlap blocks.
 * Asynchronous on `stream`; allocates nothing.  BF_ERR_INVALID for bad
 * sizes, ranges or host pointers; BF_ERR_UNSUPPORTED for k > 32. */
bf_status bf_sketch_products(const bf_sketch_desc *desc, const unsigned long long *c_fixed,
                             const void *blocks, void *out, cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * Factor files.  Constructing a factorization (Sec. 3) costs far more than
 * applying it, so a factorization is stored once and planned again later.
 * A factor file is a 64-byte header -- magic "BFLYFAC", format version (1),
 * dtype, L, leaf, r, payload size, the CRC-32 of the payload and the CRC-32
 * of the header's first 44 bytes -- followed by the arrays of bf_factors in
 * canonical order (VL, H[0..h-1], S, G[0..h-1], UL; S real in the dtype's
 * precision and zero-padded to a multiple of 8 bytes).  The writer is the
 * Python binding's `bf_factor_file_save`.  CRC-32 here is ISO-HDLC / IEEE
 * 802.3 (reflected polynomial 0xEDB88320; "123456789" -> 0xCBF43926).
 * ------------------------------------------------------------------------- */

/* Reads and verifies a factor file without creating anything: BF_OK and its
 * shape in *desc (nrhs_max = 0) and dtype in *dtype (either may be NULL);
 * BF_ERR_CORRUPT for a wrong magic, a header or payload checksum that does
 * not match, a shape outside the compiled limits, or a file shorter or longer
 * than its header says; BF_ERR_UNSUPPORTED for another format version;
 * BF_ERR_INVALID if the file cannot be opened.  Host only, no CUDA call. */
bf_status bf_factor_file_check(const char *path, bf_desc *desc, int *dtype);

/* bf_plan_create from a factor file (verified as by bf_factor_file_check
 * before any CUDA call; the payload is read into a host buffer that is freed
 * before returning).  Errors as bf_factor_file_check, then as bf_plan_create. */
bf_status bf_plan_create_from_file(bf_plan *plan, const char *path, int nrhs_max, cudaStream_t stream);

/* Running CRC-32 of `bytes` bytes (start from crc = 0), the checksum of the
 * factor files. */
unsigned int bf_crc32(const void *data, size_t bytes, unsigned int crc);

/* Static text for a status code. */
const char *bf_status_string(bf_status status);

#ifdef __cplusplus
}
#endif

#endif /* BFLY_H */
