/*
 * crsolve.h -- C ABI of a GB300 (sm_103a) solver for Hermitian positive
 * definite block-tridiagonal linear systems by classic cyclic reduction.
 *
 * The system (Sec. 1, eq. Axb and eq. Data):
 *     [ A_1  B_1^H                ] [x_1]   [y_1]
 *     [ B_1  A_2   B_2^H          ] [x_2] = [y_2]
 *     [      ...   ...    ...     ] [...]   [...]
 *     [            B_{N-1} A_N    ] [x_N]   [y_N]
 * with A_j, B_j complex m x m and x_j, y_j complex m x k.  The method reduces
 * the even-indexed half by the block formulas of Sec. 2 (eq. Formulas, with
 * the boundary auxiliaries B_0 = B_N = 0, A_0 = A_{N+1} = I), forms every
 * Hermitian product through a Cholesky factor as Sec. 4 prescribes, recurses
 * until one block is left (solved by Cholesky), and recovers the odd unknowns
 * by back-substitution from the odd block rows of eq. Axb.  A Cholesky pivot
 * that is not > 0 reports the matrix as not positive definite (Sec. 2,
 * "Determination of Positive Definiteness").
 *
 * Conventions shared by every entry point
 *   - Element type crsolve_z: interleaved complex double, 16 bytes, the same
 *     bytes as torch.complex128, numpy complex128 and cuDoubleComplex.
 *   - Layouts, all row-major and contiguous:
 *       A [N][m][m]   only the lower triangle of each A_j is read, and only
 *                     the real part of its diagonal;
 *       B [N-1][m][m] B_j sits at block position (j+1, j);
 *       y, x [N][m][k].
 *   - Device pointers must be 16-byte aligned device memory of the current
 *     device.  The library never retains A, B or y beyond the stream work
 *     that a call enqueues.
 *   - Every call is asynchronous on the given CUDA stream (NULL = legacy
 *     default stream) unless stated otherwise.  Argument errors are found on
 *     the host, return a negative code and enqueue nothing.
 *   - Breakdown (not positive definite) is found on the device; it is read
 *     back by crsolve_info_get.  After a breakdown, crsolve_solve and
 *     crsolve_backward write NaN into x / gy.
 *   - Device memory: the library allocates none for the plan.  The caller
 *     asks for the workspace size, allocates it (e.g. a torch tensor) and
 *     binds it; the plan owns its contents until crsolve_destroy.
 *   - CUDA graphs: crsolve_factor and crsolve_solve of a CRSOLVE_FP64 plan
 *     only enqueue kernels and memsets on the stream and can be captured;
 *     make the plan's first factor call outside the capture (it sets kernel
 *     attributes).  Mixed-precision plans synchronise and cannot be captured.
 *   - Tracing: every call and every reduction level is an NVTX range.
 */
#ifndef CRSOLVE_H
#define CRSOLVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } crsolve_z;
typedef struct crsolve_plan_s *crsolve_plan;

enum crsolve_status {
    CRSOLVE_OK = 0,
    CRSOLVE_NOT_PD = 1,          /* a Cholesky pivot was not > 0 (or NaN) */
    CRSOLVE_EINVAL = -1,         /* bad argument: size, null or misaligned pointer */
    CRSOLVE_ENOMEM = -2,         /* workspace missing or too small */
    CRSOLVE_ECUDA = -3,          /* a CUDA runtime call failed */
    CRSOLVE_ETIMEOUT = -4,       /* a bounded device-side wait gave up */
    CRSOLVE_ENOTFACTORED = -5,   /* solve/backward before a factor */
    CRSOLVE_EUNSUPPORTED = -6    /* m or k outside the supported range */
};

enum crsolve_precision {
    CRSOLVE_FP64 = 0,            /* every step in FP64 */
    CRSOLVE_MIXED = 1            /* FP32 factor + FP64 residual and refinement */
};

/* plan flags */
#define CRSOLVE_PLAN_HOST_STAGING 1u  /* workspace also holds device copies of A, B, y, x
                                         for crsolve_solve_host */
#define CRSOLVE_PLAN_ALG1 2u          /* the paper's own method, Algorithm 1 (Sec. 3) */
#define CRSOLVE_PLAN_FP64_RESIDUAL 4u /* mixed precision: residuals and products on the FP64
                                         pipe even where the tensor-core splitting applies */

/*
 * Plans with CRSOLVE_PLAN_ALG1 run the paper's Algorithm 1 instead of classic
 * reduction: every level splits each system into its odd half (U, E, u) and
 * its even half (V, F, v) of eq. Formulas and recurses on both, down to
 * single m x m blocks solved by Cholesky; there is no back-substitution.
 * Level l holds 2^l systems of N/2^l blocks, so every level factors all N
 * diagonal blocks (N log2 N block factorisations in total against N for
 * classic reduction) and the workspace keeps log2 N + 1 levels of factors.
 * N must be a power of two (Algorithm 1 assumes it) and precision
 * CRSOLVE_FP64; otherwise crsolve_plan_create returns CRSOLVE_EUNSUPPORTED.
 * crsolve_info: level = recursion depth of the first breakdown (log2 N = the
 * single blocks), orig_block = the smallest failing original block at that
 * depth, block = its 1-based position among the N blocks of that depth (the
 * split systems in order, each split putting the odd half first).
 * crsolve_factor, crsolve_solve, crsolve_backward and crsolve_solve_host work
 * unchanged on such plans.
 */

/* Largest block size m and right-hand-side width k the kernels accept. */
#define CRSOLVE_MAX_M 64
#define CRSOLVE_MAX_K 4096

typedef struct {
    int32_t status;     /* CRSOLVE_OK or CRSOLVE_NOT_PD */
    int32_t level;      /* 0-based reduction level of the first breakdown */
    int64_t block;      /* 1-based block index within that level */
    int64_t orig_block; /* 1-based index of that block in the original system
                           (block * 2^level: even block 2j at one level is block
                           j at the next) */
} crsolve_info;

/*
 * crsolve_plan_create -- describe one system shape (host only, no CUDA call).
 *   N >= 1 blocks of size 1 <= m <= CRSOLVE_MAX_M; right-hand sides of width
 *   up to kmax (1 <= kmax <= CRSOLVE_MAX_K); precision from crsolve_precision;
 *   flags from CRSOLVE_PLAN_*.  The plan is tied to the current device.
 * Returns CRSOLVE_OK, CRSOLVE_EINVAL or CRSOLVE_EUNSUPPORTED.
 */
int crsolve_plan_create(int64_t N, int32_t m, int32_t kmax, int32_t precision,
                        uint32_t flags, crsolve_plan *out_plan);

/* Bytes of device workspace the plan needs (per-level factors, the reduced
 * systems, scratch and, with CRSOLVE_PLAN_HOST_STAGING, input/output copies). */
int crsolve_workspace_bytes(crsolve_plan p, size_t *bytes);

/* Bind caller-owned device memory (256-byte aligned, >= crsolve_workspace_bytes)
 * to the plan.  The caller frees it after crsolve_destroy. */
int crsolve_set_workspace(crsolve_plan p, void *dev_ptr, size_t bytes);

/*
 * crsolve_plan_keep_levels -- trade compute for memory (classic FP64 plans;
 * call before crsolve_set_workspace).  The plan's memory is split in two:
 *   workspace  the factors (L, 1/diag L, Z = [P | Q]) of the fine levels
 *              0 .. keep-1 and the reduced system (A^(keep), B^(keep)) of
 *              level keep, plus the breakdown status;
 *   scratch    the factors of the coarse levels keep .. L, the right-hand
 *              sides and solutions of every level during a solve, and the
 *              CTA-boundary buffers and their arrival counters (zeroed by
 *              each factor and solve call; crsolve_scratch_bytes,
 *              crsolve_set_scratch).
 * Level l has ceil(N_l / 2) odd blocks, so the workspace holds about
 * 1 - 2^-keep of the factor storage, and rebuilding the coarse levels costs
 * about 2^-keep of a factorisation.  Factor, solve, backward and solve_host
 * calls need the scratch bound; between calls it may be unbound
 * (crsolve_set_scratch(p, NULL, 0)) and its memory reused.  Binding scratch
 * (any pointer, even the same one) marks the coarse factors as lost: the next
 * crsolve_solve or crsolve_backward first re-factors levels keep .. L from the
 * stored level-keep system (the recursion of Sec. 2 "Formulation of the
 * Method" restarted at level keep), which is deterministic, so results are
 * bit-identical to an unsplit plan's.  keep = 0 keeps no factors: the
 * re-factorisation starts from the A and B given to crsolve_factor, which must
 * then stay valid and unchanged (after crsolve_solve_host, whose staged A and B
 * live in the scratch, that gives CRSOLVE_ENOTFACTORED).  keep = -1 (the
 * default) keeps everything in the workspace and uses no scratch.
 * Returns CRSOLVE_EINVAL (keep < -1, or workspace or scratch already bound) or
 * CRSOLVE_EUNSUPPORTED (Algorithm 1 or mixed-precision plans).
 */
int crsolve_plan_keep_levels(crsolve_plan p, int32_t keep);

/* Bytes of scratch a plan split by crsolve_plan_keep_levels needs (0 otherwise). */
int crsolve_scratch_bytes(crsolve_plan p, size_t *bytes);

/* Bind caller-owned device memory (256-byte aligned, >= crsolve_scratch_bytes)
 * as the scratch of a split plan, or unbind it with dev_ptr = NULL.  Returns
 * CRSOLVE_EINVAL on an unsplit plan, CRSOLVE_ENOMEM if bytes is too small. */
int crsolve_set_scratch(crsolve_plan p, void *dev_ptr, size_t bytes);

/*
 * crsolve_factor -- the reduction sweep of Sec. 2 on device data.
 *   A [N][m][m], B [N-1][m][m] (B may be NULL iff N == 1).  For every level it
 *   factors the odd diagonal blocks (Cholesky with breakdown test), forms
 *   P_i = L_i^{-1} B_{i-1}, Q_i = L_i^{-1} B_i^H and the half-size even system
 *   V_j = A_{2j} - Q_{2j-1}^H Q_{2j-1} - P_{2j+1}^H P_{2j+1},
 *   F_j = -Q_{2j+1}^H P_{2j+1} (eq. Formulas with the Sec. 4 product rule),
 *   and keeps L, P, Q of every level in the workspace for later solves.
 *   On a classic FP64 plan it enqueues only kernels and memsets on the
 *   stream: one kernel per level, plus a fix-up kernel for the CTA-boundary
 *   blocks on levels of more than four CTAs per SM.
 * Returns CRSOLVE_OK once enqueued; breakdown is reported by crsolve_info_get.
 */
int crsolve_factor(crsolve_plan p, const crsolve_z *A, const crsolve_z *B, void *stream);

/*
 * crsolve_solve -- x = A^{-1} y with the stored factorisation.
 *   y, x [N][m][k] device, 1 <= k <= kmax, x must not alias y.  Down sweep:
 *   r_i = L_i^{-1} y_i, v_j = y_{2j} - Q_{2j-1}^H r_{2j-1} - P_{2j+1}^H r_{2j+1}
 *   (eq. Formulas); up sweep: x_i = L_i^{-H}(r_i - P_i x_{i-1} - Q_i x_{i+1}).
 * Returns CRSOLVE_ENOTFACTORED before the first crsolve_factor.
 */
int crsolve_solve(crsolve_plan p, int32_t k, const crsolve_z *y, crsolve_z *x, void *stream);

/*
 * crsolve_backward -- adjoint of x = A^{-1} y for a real loss L.
 *   Given x (the solve's result) and gx = dL/dx (PyTorch's complex gradient
 *   convention, dL/dRe + i dL/dIm), writes
 *     gy  = A^{-1} gx   (a re-solve with the stored factors; A is Hermitian),
 *     gA_j = -1/2 (gy_j x_j^H + x_j gy_j^H)   (projected onto Hermitian
 *            matrices: the gradient for Hermitian perturbations of A_j),
 *     gB_j = -(gy_{j+1} x_j^H + x_{j+1} gy_j^H)   (B_j enters at (j+1,j) and
 *            as B_j^H at (j,j+1)).
 *   gA [N][m][m] and gB [N-1][m][m] may be NULL.  The paper has no adjoint;
 *   these are the derivatives of the system of eq. Axb.
 */
int crsolve_backward(crsolve_plan p, int32_t k, const crsolve_z *x, const crsolve_z *gx,
                     crsolve_z *gy, crsolve_z *gA, crsolve_z *gB, void *stream);

/*
 * crsolve_solve_host -- factor and solve with HOST buffers: copies A, B, y
 * from host memory (pinned for full speed) into the plan's staging area,
 * factors, solves, copies x back to host memory and synchronises the stream.
 * For classic plans with N > 1 the copies run on a second stream owned by the
 * plan and overlap the kernels: the level-0 factor starts range by range as
 * the rows of A and B it reads arrive, followed after each range by the
 * chunks of levels 1-3 whose rows are complete; y is copied while the rest is
 * factored, and x is copied back range by range behind the level-0 up sweep.  x is bit-identical to crsolve_factor + crsolve_solve.  The
 * factorisation is FP64 for every plan: on a CRSOLVE_MIXED plan, later
 * crsolve_solve calls use it (FP64) until the next crsolve_factor.
 * Needs a plan created with CRSOLVE_PLAN_HOST_STAGING.  Returns CRSOLVE_OK or
 * CRSOLVE_NOT_PD (then x holds NaN), or a negative error.
 */
int crsolve_solve_host(crsolve_plan p, int32_t k, const crsolve_z *A_host,
                       const crsolve_z *B_host, const crsolve_z *y_host, crsolve_z *x_host,
                       void *stream);

/* Synchronises the stream and reports the factorisation's breakdown status. */
int crsolve_info_get(crsolve_plan p, crsolve_info *out, void *stream);

/* Frees the host-side plan (not the caller's workspace). */
int crsolve_destroy(crsolve_plan p);

/* Static description of a status code. */
const char *crsolve_strerror(int code);

/* ---- batched: many independent systems in one persistent launch ---- */

typedef struct crsolve_batch_s *crsolve_batch;

/*
 * crsolve_batch_create -- describe nsys independent systems (host only apart
 * from reading the device properties).  System i has N[i] >= 1 blocks of
 * size 1 <= m[i] <= CRSOLVE_MAX_M and k[i] >= 1 right-hand sides.  Inputs
 * are packed back to back in system order: system i's A starts at element
 * offA[i] = sum_{j<i} N_j m_j^2 of one A array, its B at offB[i] =
 * sum_{j<i} (N_j - 1) m_j^2, its y and x at offY[i] = sum_{j<i} N_j m_j k_j
 * (crsolve_batch_offsets reports them).  The systems are independent (the
 * block formulas of Sec. 2 never couple two systems); each is solved by the
 * same classic cyclic reduction as crsolve_factor + crsolve_solve, with
 * bit-identical arithmetic.
 */
int crsolve_batch_create(int32_t nsys, const int64_t *N, const int32_t *m, const int32_t *k,
                         crsolve_batch *out);

/* Tile shape of block-size class mt for this batch (odd blocks per chunk of
 * the factor and solve steps, right-hand-side columns per chunk); before
 * crsolve_batch_set_workspace.  CRSOLVE_EINVAL if out of range or if the
 * kernel would not fit in shared memory. */
int crsolve_batch_tile_set(crsolve_batch b, int32_t mt, int32_t nb_factor, int32_t nb_solve, int32_t kc);

/* Workspace size: one slot per persistent CTA (as many as fit on the device,
 * at most nsys, and at most what fits in max_bytes when max_bytes > 0) plus
 * per-system descriptors and status.  Reports the slot count in *nslots. */
int crsolve_batch_workspace_bytes(crsolve_batch b, size_t max_bytes, size_t *bytes, int32_t *nslots);

/* Bind caller-owned device memory (256-byte aligned, >= the size above). */
int crsolve_batch_set_workspace(crsolve_batch b, void *dev_ptr, size_t bytes);

/* Element offsets of every system in the packed arrays (host arrays of nsys
 * entries, any may be NULL) and totals[3] = elements of A, B and y/x. */
int crsolve_batch_offsets(crsolve_batch b, int64_t *offA, int64_t *offB, int64_t *offY, int64_t *totals);

/* Factor and solve every system: one persistent kernel launch on the stream
 * (plus two memsets).  A, B, y, x are the packed device arrays; x must not
 * alias y.  Per-system breakdown is read with crsolve_batch_info. */
int crsolve_batch_solve(crsolve_batch b, const crsolve_z *A, const crsolve_z *B, const crsolve_z *y,
                        crsolve_z *x, void *stream);

/* Same as crsolve_batch_solve, through a CUDA graph captured on the first
 * call (and again whenever the pointers change) and replayed on the stream. */
int crsolve_batch_graph_launch(crsolve_batch b, const crsolve_z *A, const crsolve_z *B, const crsolve_z *y,
                               crsolve_z *x, void *stream);

/* Synchronises the stream and writes nsys breakdown records into out. */
int crsolve_batch_info(crsolve_batch b, crsolve_info *out, void *stream);

int crsolve_batch_destroy(crsolve_batch b);

/*
 * crsolve_solve_noalloc -- factor and solve one system with no device
 * allocation, for callers that cannot call cudaMalloc (code running where the
 * allocator is unavailable or forbidden, e.g. a host callback, a
 * pre-allocated real-time loop, or a plugin that must not grow the device
 * footprint after start-up).  The paper has no counterpart; this is the same
 * classic cyclic reduction as crsolve_factor + crsolve_solve.
 *   The caller passes A [N][m][m], B [N-1][m][m] (NULL iff N == 1), y and x
 *   [N][m][k] in device memory, as for crsolve_factor / crsolve_solve.  All
 *   intermediates live in one fixed 32 MiB device array inside this library
 *   (held by every GPU that loads the library until the process exits); a
 *   system whose intermediates exceed it returns CRSOLVE_ENOMEM and enqueues
 *   nothing (about N * (5.5 m^2 + 3.5 m k) * 16 bytes must fit, e.g. N up to
 *   ~4500 for m = 8, k = 4).
 *   Every call looks up the array's device address (cudaGetSymbolAddress,
 *   with the caller's device current) and sets the shared-memory limits of
 *   its kernels; nothing is cached between calls, so a device reset or
 *   another context of the device never leaves a stale address.  The first
 *   call on a device also loads the library's kernels onto it: make it
 *   before any stream capture.  All calls share the array and it keeps the
 *   last call's contents, so calls that overlap on the GPU race: serialise
 *   them.  After a breakdown x holds NaN.  With info != NULL
 *   the call synchronises the stream and reports the breakdown status there;
 *   with info == NULL it is asynchronous.
 */
int crsolve_solve_noalloc(int64_t N, int32_t m, int32_t k, const crsolve_z *A, const crsolve_z *B,
                          const crsolve_z *y, crsolve_z *x, crsolve_info *info, void *stream);

/* ---- instrumentation (the paper has no counterpart; used by the benchmark) ---- */

enum crsolve_kernel_kind {
    CRSOLVE_K_FACTOR_ODD = 0,      /* Cholesky + P, Q + Z^H Z of a level's odd blocks, and
                                      the next level's blocks inside each CTA */
    CRSOLVE_K_FACTOR_FIX = 1,      /* next level's blocks on CTA boundaries */
    CRSOLVE_K_SOLVE_DOWN_ODD = 2,  /* r = L^{-1} y, Z^H r and the next level's right-hand
                                      side inside each CTA */
    CRSOLVE_K_SOLVE_DOWN_FIX = 3,  /* next level's right-hand side on CTA boundaries */
    CRSOLVE_K_SOLVE_UP = 4,        /* back-substitution of a level */
    CRSOLVE_K_ADJOINT = 5,         /* gA, gB outer products */
    CRSOLVE_K_NANFILL = 6,         /* NaN fill of gA / gB after a breakdown */
    CRSOLVE_K_RESIDUAL = 7,        /* mixed precision: FP64 residual y - A x */
    CRSOLVE_K_CONVERT = 8,         /* mixed precision: FP64 <-> FP32 copies */
    CRSOLVE_K_UPDATE = 9,          /* mixed precision: x += d and norms */
    CRSOLVE_K_ALG1_BORDER = 10,    /* Algorithm 1: auxiliary border blocks of the level buffers */
    CRSOLVE_K_ALG1_MERGE = 11      /* Algorithm 1: merge of the two base solutions */
};

typedef struct {
    int32_t kind;    /* crsolve_kernel_kind */
    int32_t level;   /* reduction level (0 for kernels outside the sweep) */
    int64_t units;   /* odd blocks the launch processed (CTA boundaries for the fix-ups) */
    float ms;        /* duration between CUDA events recorded around the launch */
} crsolve_kernel_time;

/* With enable != 0, every kernel the plan launches is bracketed by CUDA events
 * recorded on the launch stream; records accumulate until read.  Not for use
 * inside stream capture. */
int crsolve_timing_enable(crsolve_plan p, int32_t enable);

/* Waits for the recorded events and returns up to cap records (oldest first)
 * in out, the number available in *count; then clears the records. */
int crsolve_timing_read(crsolve_plan p, crsolve_kernel_time *out, int32_t cap, int32_t *count);

/*
 * Mixed precision (plans created with CRSOLVE_MIXED).  The levels of the
 * reduction with more than 2 blocks are factored and solved in FP32; the two
 * coarsest levels, the breakdown decision, the residuals and products of the
 * refinement and the refinement itself are FP64.  The refinement is
 * preconditioned conjugate gradients per right-hand-side column (A is
 * Hermitian positive definite) with the FP32 solve as preconditioner, the
 * CG variant of the mixed-precision iterative refinement of Carson and Higham
 * (SIAM J. Sci. Comput. 39, 2017); it stops when the last relative
 * correction is below 1e-11, a tenth of the stated bound 1e-10, or, late in
 * the run (correction <= 1e-8, contraction <= 1e-2), when the observed
 * contraction times the last correction is below 1e-12; when the first
 * correction shows a condition number above about 1e3, the first stop is
 * followed by one restart from the true residual.  For m > 32 the FP64-
 * accurate residuals and products come from exact splitting on the tensor
 * cores (see crsolve_residual, method CRSOLVE_RESIDUAL_SPLIT) unless the plan
 * was created with CRSOLVE_PLAN_FP64_RESIDUAL, and the FP32 factorisation
 * keeps L^{-1} in place of L, so that the FP32 sweeps are complex matrix
 * products instead of triangular substitutions.  In this mode crsolve_factor and
 * crsolve_solve synchronise the stream, and A and B must stay valid and
 * unchanged until the plan is re-factored or destroyed (the residual reads
 * them).  A breakdown in the FP32 levels is re-decided by an FP64
 * factorisation, so the flags are always the FP64 ones.  The iteration hands
 * over to the FP64 path (factor + solve) when it does not contract, loses
 * positive curvature, or when the steps still needed at the observed rate
 * would cost more than that path.
 * crsolve_mixed_stats reports the last solve: FP64-accurate residuals and
 * products computed (1 + CG steps), delta = the last relative correction
 * (largest over the columns of |alpha p|_inf / |x|_inf), rho = the observed
 * contraction per step, and whether the FP64 path was used instead.
 */
int crsolve_mixed_stats(crsolve_plan p, int32_t *iterations, double *delta, double *rho, int32_t *fp64_fallback);

/*
 * The preconditioner of the mixed-precision form alone: z = A~^{-1} r, one
 * solve with the FP32 levels and the FP64 coarse levels of the factorisation
 * (Sec. 2 eq. Formulas, the down and up sweeps, in FP32 on every level with
 * more than 2 blocks), without refinement; for users who run their own
 * Krylov iteration around it.  r and z: device [N][m][k] complex128, k <=
 * kmax, 16-byte aligned, may be the same buffer (r is read first).  Enqueued
 * on `stream`, no synchronisation.  The accuracy is that of FP32 arithmetic
 * (about kappa * 2^-24 relative).  CRSOLVE_EUNSUPPORTED for plans other than
 * CRSOLVE_MIXED, for plans without FP32 levels (N <= 2), and after an FP32
 * breakdown (the plan then holds only the FP64 factorisation);
 * CRSOLVE_ENOTFACTORED before crsolve_factor.
 */
int crsolve_mixed_precondition(crsolve_plan p, int32_t k, const crsolve_z *r, crsolve_z *z, void *stream);

/*
 * crsolve_residual -- r = y - A x for the block-tridiagonal A of eq. Axb
 * (A_j Hermitian, read from its lower triangle and the real part of its
 * diagonal; B_j at block (j+1, j), B_j^H at (j, j+1)), the residual of the
 * iterative refinement in the mixed-precision form.  Layouts as for
 * crsolve_factor / crsolve_solve: A [N][m][m], B [N-1][m][m] (NULL iff
 * N == 1), x, y, r [N][m][k], all device memory, 16-byte aligned; r must not
 * alias x (it may alias y).
 *   method CRSOLVE_RESIDUAL_FP64: FP64 fused multiply-adds; no workspace;
 *   asynchronous.
 *   method CRSOLVE_RESIDUAL_SPLIT: every product exact on the BF16 tensor
 *   cores (error-free splitting of Ozaki, Ogita, Oishi and Rump, 2012: a
 *   matrix entry cut into ten 6-bit integer slices on a per-row binary grid
 *   of 60 bits, an x entry into nine on a per-column grid of 54 bits, slice
 *   products with i + j <= 11 accumulated exactly in FP32 in tensor memory),
 *   then y - A x formed exactly in 128-bit integers and rounded once; the
 *   dropped slice products and the grids add less than about 2^-50 K
 *   max|row of A| max|column of x| (K = 6m), within the error bound of an
 *   FP64 dot product, and, unlike an FP64 residual, nothing is rounded per
 *   product or per sum.  Needs a
 *   256-byte aligned device workspace of crsolve_residual_workspace_bytes;
 *   synchronises the stream and returns CRSOLVE_ETIMEOUT if a bounded wait of
 *   the tensor-core pipeline gave up.  The paper has no counterpart.
 *   method CRSOLVE_RESIDUAL_SPLIT_IMAGE: the same result, bit for bit, with
 *   the matrix slices first written to the workspace in the tensor cores'
 *   shared-memory layout (about 0.94 MiB per block row) and then copied in by
 *   bulk copies; the mixed-precision form does this once per factorisation
 *   and reuses the slices for every residual of its refinement.
 */
enum { CRSOLVE_RESIDUAL_FP64 = 0, CRSOLVE_RESIDUAL_SPLIT = 1, CRSOLVE_RESIDUAL_SPLIT_IMAGE = 2 };
int crsolve_residual_workspace_bytes(int64_t N, int32_t m, int32_t k, int32_t method, size_t *bytes);
int crsolve_residual(int64_t N, int32_t m, int32_t k, const crsolve_z *A, const crsolve_z *B, const crsolve_z *x,
                     const crsolve_z *y, crsolve_z *r, int32_t method, void *workspace, size_t workspace_bytes,
                     void *stream);

/*
 * crsolve_peak_probe -- measured arithmetic rate of the current device, for
 * rooflines (the paper has no counterpart).  kind CRSOLVE_PROBE_FP64_FMA
 * times independent FP64 fused multiply-add chains (the pipe that bounds the
 * FP64 path), CRSOLVE_PROBE_FP32_FMA the FP32 ones; no memory traffic.
 * Writes the rate in GFLOP/s (2 flop per FMA) to *gflops and, when not NULL,
 * the FMA lanes per SM per clock cycle (clock-independent) to *fma_per_clk_sm
 * and the SM clock the kernel ran at to *sm_mhz.  Runs two kernels (a short
 * warm-up and the timed one, ~0.1 s) on the stream and synchronises it.
 * CRSOLVE_EINVAL for a NULL gflops or an unknown kind.
 */
enum { CRSOLVE_PROBE_FP64_FMA = 0, CRSOLVE_PROBE_FP32_FMA = 1 };
int crsolve_peak_probe(int32_t kind, double *gflops, double *fma_per_clk_sm, double *sm_mhz, void *stream);

/*
 * crsolve_check_bounded_wait -- exercises the bounded mbarrier wait of the
 * tensor-core kernels on its own (the paper has no counterpart): one CTA
 * waits, with a limit of max_polls polls (and about two seconds), on an
 * mbarrier that nothing arrives at.  Returns CRSOLVE_ETIMEOUT when the wait
 * gave up as it should, CRSOLVE_OK if it completed.  workspace: 4 bytes of
 * device memory.  Synchronises the stream.
 */
int crsolve_check_bounded_wait(int32_t max_polls, void *workspace, void *stream);

/* Kernels this plan has launched since it was created. */
int crsolve_launch_count(crsolve_plan p, int64_t *count);

/*
 * Tile shape of block-size class mt (4, 8, 16, 32 or 64; a plan with block
 * size m uses the smallest class >= m) of the FP64 kernels: odd blocks per
 * CTA of the factor and of the solve kernels, right-hand-side columns per
 * solve CTA (narrowed automatically on small levels), and threads per CTA of
 * the factor and of the solve kernels (multiples of 32, at most 256).
 * Process-wide, for later launches.  crsolve_tile_set returns CRSOLVE_EINVAL
 * for a shape that is out of range or does not fit in the current device's
 * shared memory.
 */
int crsolve_tile_set(int32_t mt, int32_t nb_factor, int32_t nb_solve, int32_t kc, int32_t threads,
                     int32_t threads_solve);
int crsolve_tile_get(int32_t mt, int32_t *nb_factor, int32_t *nb_solve, int32_t *kc, int32_t *threads,
                     int32_t *threads_solve);
/* The same for the FP32 levels of the mixed-precision form (their own table;
 * for mt = 64 the factor runs with exactly 256 threads, and the solve fields
 * nb_solve, kc, threads_solve are stored but not used: that class keeps
 * L^{-1} and solves with fixed-shape product kernels, one odd block and a
 * column chunk of 8, 16 or 32 per work item: by k, narrower on levels with
 * fewer odd blocks than SMs). */
int crsolve_tile_set_mixed(int32_t mt, int32_t nb_factor, int32_t nb_solve, int32_t kc, int32_t threads,
                           int32_t threads_solve);
int crsolve_tile_get_mixed(int32_t mt, int32_t *nb_factor, int32_t *nb_solve, int32_t *kc, int32_t *threads,
                           int32_t *threads_solve);

/* Number of levels of the plan (floor(log2 N) + 1) and the level sizes; with
 * CRSOLVE_PLAN_ALG1, log2 N + 1 levels of N blocks each (2^l systems of N/2^l). */
int crsolve_plan_levels(crsolve_plan p, int32_t *nlev, int64_t *sizes /* [nlev] or NULL */);

/*
 * Bounds-checked builds (compiled with CRSOLVE_DEBUG_BOUNDS, the library
 * libcrsolve_debug.so; the paper has no counterpart).  Every global-memory
 * index of the level kernels (and of the tensor-core residual) is checked
 * against the array extents implied by the level sizes (A [N_l][m][m],
 * B [N_l-1][m][m], L [no][m][m], Z [no][m][2m], y, x [N_l][m][k], ...); an
 * out-of-range index is skipped (a load reads zero) and the smallest record
 * (level << 56 | array << 48 | index, array numbers as in crs::DbgArray) is
 * kept in a word of the plan's (or batch's) workspace, cleared by every
 * crsolve_factor / crsolve_solve_host / batch launch.  These calls
 * synchronise the stream and write that record (all ones: no out-of-range
 * access) to *record.  Release builds return CRSOLVE_EUNSUPPORTED.
 */
int crsolve_debug_bounds(crsolve_plan p, uint64_t *record, void *stream);
int crsolve_batch_debug_bounds(crsolve_batch b, uint64_t *record, void *stream);

/*
 * crsolve_debug_level_system -- device pointers of the reduced system
 * (A^(l), B^(l)) of level l >= 1 inside the bound workspace, for tests that
 * compare each level with the oracle.  Valid after crsolve_factor.
 */
int crsolve_debug_level_system(crsolve_plan p, int32_t level, const crsolve_z **A_l,
                               const crsolve_z **B_l);

#ifdef __cplusplus
}
#endif
#endif /* CRSOLVE_H */
