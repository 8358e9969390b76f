/*
 * rhif.h -- C ABI of the GB300 implementation of the recursively preconditioned
 * hierarchical interpolative factorization (PHIF) of Feliu-Faba, Ho and Ying.
 *
 * Problem (Sec. 1, Eqs. 1.1-1.2): A u = f, A sparse SPD from the five-point
 * (2D) or seven-point (3D) finite-difference discretisation of
 * -div(a grad u) + b u = f on the unit square/cube with zero Dirichlet data.
 * The library builds F ~= A (Sec. 3, Eqs. 3.1-3.3), applies F^{-1}, and runs
 * PCG with F^{-1} as the preconditioner (Sec. 4).
 *
 * Conventions for every entry point:
 *  - A grid has n[i] interior nodes along axis i (x first), h_i = 1/(n[i]+1).
 *    DOF index of interior node (i,j,k) (0-based) is i + n0*(j + n1*k).
 *  - Unless stated otherwise every array pointer is a DEVICE pointer owned by
 *    the caller; the library never frees caller memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  All work is stream-ordered on it; calls that return host
 *    results (statistics, iteration counts) synchronise that stream.
 *  - Return value: RHIF_OK (0) or a negative RHIF_ERR_* code; no exception or
 *    trap crosses the ABI.  rhif_error_string() names a code and
 *    rhif_last_error_detail() gives a one-line description of the most recent
 *    failure on the calling thread.
 *  - A handle must not be used concurrently from two streams.
 */
#ifndef RHIF_H
#define RHIF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  RHIF_OK = 0,
  RHIF_ERR_BAD_ARG = -1,        /* null pointer, bad size, CSR outside the stencil pattern */
  RHIF_ERR_NOT_SPD = -2,        /* a Cholesky pivot <= 0 or NaN (Remark 2.1: SPD lost) */
  RHIF_ERR_NOT_CONVERGED = -3,  /* PCG hit maxit before rtol */
  RHIF_ERR_TIMEOUT = -4,        /* a bounded device wait gave up */
  RHIF_ERR_OOM = -5,            /* device allocation failed */
  RHIF_ERR_CUDA = -6,           /* any other CUDA runtime error */
  RHIF_ERR_CHECK = -7           /* a self-check found a violated invariant (detail says which) */
};

/* Precision of the factor.  RHIF_FP64: every step in FP64.  The mixed
 * precisions store and compute the factor in FP32 (the application of F^{-1}
 * too; PCG's vectors, SpMV and dots stay FP64) and differ only in the
 * operands of the tensor-core Schur tiles of fronts eliminated with the
 * many-CTA schedule (Sec. 2.1 Schur update; in practice the 3D levels >= 1):
 * RHIF_MIXED_FP32 splits each value into two TF32 parts (three products,
 * about FP32 accuracy), RHIF_MIXED_TF32 uses one TF32 product, and
 * RHIF_MIXED_BF16 one BF16 product, all accumulated in FP32. */
enum { RHIF_FP64 = 0, RHIF_MIXED_FP32 = 1, RHIF_MIXED_TF32 = 2, RHIF_MIXED_BF16 = 3 };
/* operand kinds of rhif_tc_gemm_check */
enum { RHIF_TC_TF32X3 = 0, RHIF_TC_TF32 = 1, RHIF_TC_BF16 = 2 };
enum { RHIF_PRECOND_NONE = 0, RHIF_PRECOND_BLOCK = 1, RHIF_PRECOND_DIAG = 2 };
/* operations of rhif_apply: F^{-1}, F, G^{-1}, G^{-T} with F = G G^T (Eq. 3.3) */
enum { RHIF_SOLVE = 0, RHIF_MATVEC = 1, RHIF_HALF = 2, RHIF_HALF_T = 3 };

typedef struct {
  int dim;      /* 2 or 3 */
  int n[3];     /* interior nodes per axis (n[2] ignored when dim == 2) */
} rhif_grid;

/* Sparse matrix in CSR form, device memory, caller-owned.  Row r holds
 * col[rowptr[r] .. rowptr[r+1]) with values val[...].  The pattern must be the
 * grid stencil (diagonal plus grid neighbours) and the values symmetric. */
typedef struct {
  int64_t nrows;
  int64_t nnz;
  const int64_t* rowptr;
  const int32_t* col;
  const double* val;
} rhif_csr;

typedef struct {
  int precision;      /* RHIF_FP64 (default), RHIF_MIXED_FP32, _TF32 or _BF16 */
  /* precondition: local preconditioner C_l applied to every separator group
   *   before skeletonization.  1 = block Jacobi by the Cholesky factor of the
   *   group's diagonal block (PHIF, Sec. 2.3; default); 0 = none (plain HIF,
   *   C_l = I); 2 = diagonal, C_g = diag(A_gg)^{-1/2} (the cheaper local
   *   preconditioner the concluding section names in place of block
   *   Cholesky).  Other values: RHIF_ERR_BAD_ARG. */
  int precondition;
  int edge_skel_3d;   /* 3D only: also precondition and skeletonize edges (Remark 3.1) */
  /* Scheduling only (the result does not depend on them beyond rounding order):
   * big_front: front order (interior + boundary DOFs of a cell) from which a
   *   level's fronts are eliminated by panel / trailing-tile launches over many
   *   CTAs instead of one CTA per front; 0 = library default (384), < 0 = never.
   * big_frame: frame order (boundary DOFs of a cell) from which the block
   *   Jacobi scaling of Eq. (2.3) runs as row / column block solves over many
   *   CTAs; 0 = library default (when the frame no longer fits in shared
   *   memory, and for the FP32 factor from 96), < 0 = never. */
  int big_front;
  int big_frame;
  /* skel_cluster: CTAs (a thread-block cluster, power of two <= 16) that share
   *   the interpolative decomposition of one skeletonization unit, each holding
   *   a slice of the unit's rows.  0 = library default (one warp per unit when
   *   every unit has at most 32 DOFs, clusters only for units whose ID matrix
   *   does not fit in one CTA's shared memory, else one CTA per unit), < 0 =
   *   one CTA per unit always, 1..16 = clusters of that size always. */
  int skel_cluster;
  /* tensor_cores: FP32 factors form the Schur complements of fronts eliminated
   *   with the many-CTA schedule on the tensor cores (TF32 inputs split into
   *   a high part and a remainder: about FP32 accuracy); 0 = on (default),
   *   < 0 = off (CUDA cores).  FP64 factors always use the CUDA cores. */
  int tensor_cores;
  /* leaf_fp64: FP32 factors (precision pattern): every 2D leaf whose estimated
   *   condition number kappa_1(D A_II D) (D = diag(A_II)^{-1/2}; Hager's
   *   estimate of ||(D A_II D)^{-1}||_1 from the FP32 band factor) exceeds
   *   10^leaf_fp64 is eliminated again in FP64 arithmetic, its band, couplings
   *   and Schur complement stored rounded to FP32.  0 = default (10^6),
   *   < 0 = never, at most 30.  FP64 factors and 3D leaves ignore it; a leaf
   *   whose FP32 Cholesky broke down is still reported as NOT_SPD. */
  int leaf_fp64;
} rhif_opts;

typedef struct rhif_handle rhif_handle;

/* Fill *o with the defaults (FP64, PHIF, no 3D edge skeletonization). */
int rhif_default_opts(rhif_opts* o);

/* Number of stored entries of the finite-difference matrix of grid g. */
int64_t rhif_fd_nnz(const rhif_grid* g);

/* Finite-difference matrix of Eq. (1.1) (Sec. 3.1 five-point, Sec. 3.2
 * seven-point stencil).  a_pix: per-pixel coefficient, (n0+1)*(n1+1)[*(n2+1)]
 * values, x fastest.  The weight of a grid edge is the mean of `a` over the 2
 * (2D) or 4 (3D) pixels touching it; edges to boundary nodes add to the
 * diagonal only; entries carry the 1/h^2 factor.  b_node: per-node b (N
 * values) or NULL to use the constant b_const.  Outputs rowptr (N+1), col and
 * val (rhif_fd_nnz(g) each), caller-allocated; columns ascend within a row. */
int rhif_assemble_fd(const rhif_grid* g, const double* a_pix, const double* b_node,
                     double b_const, int64_t* rowptr, int32_t* col, double* val,
                     void* stream);

/* As rhif_assemble_fd, but from the per-pixel log-coefficient: a = exp(log_a)
 * is written to a_pix_out (one value per pixel, caller-allocated) and used for
 * the assembly.  This is the parameterization of the differentiation pattern
 * (gradient with respect to log a, see rhif_grad_logcoef). */
int rhif_assemble_fd_log(const rhif_grid* g, const double* log_a_pix, double* a_pix_out,
                         const double* b_node, double b_const, int64_t* rowptr, int32_t* col,
                         double* val, void* stream);

/* PHIF factorization F ~= A (Sec. 3): per level l = 0..L-1 cell elimination
 * (Sec. 2.1, Eq. 2.1), block Jacobi preconditioning of every separator group
 * (Sec. 2.3, Eq. 2.3) and skeletonization of every edge (2D) / face (3D) by a
 * column-pivoted-QR interpolative decomposition to relative precision `tol`
 * (Sec. 2.2, Eq. 2.2; all IDs of a level before any zeroing), then the root
 * Cholesky A_L = B_L B_L^T (Eq. 3.3).  `leaf` = m, the leaf cell width in grid
 * intervals; L is the smallest level count with 2^L m >= n_i + 1.  A is read
 * during the call only.  On success *out receives a handle owning all factor
 * storage (free with rhif_free).  Errors: BAD_ARG (pattern, sizes, leaf < 2,
 * tol < 0), NOT_SPD (with the level in the detail string), OOM, CUDA. */
int rhif_factor(const rhif_csr* A, const rhif_grid* g, int leaf, double tol,
                const rhif_opts* o, void* stream, rhif_handle** out);

/* Factor `count` independent problems (A[i] on grid g[i], same leaf, tol and
 * options) with the levels of different problems running concurrently: the
 * problems are spread over the `nstreams` CUDA streams in `streams` (problem i
 * on streams[i % nstreams]) and each stream is driven by its own host worker
 * thread.  out[i] receives the handle of problem i, or NULL if it failed; the
 * return value is the first failure's code (RHIF_OK if none).  The caller's
 * current device is used by every worker. */
int rhif_factor_batched(int count, const rhif_csr* A, const rhif_grid* g, int leaf, double tol,
                        const rhif_opts* o, void* const* streams, int nstreams,
                        rhif_handle** out);

/* Factor `count` independent problems (A[i] on grid g[i], the same
 * dimension, leaf, tol and options) as ONE merged factorization: the cells,
 * groups and units of every problem at a level form one work list, so each
 * step of a level (Sec. 2.1 cell elimination, Sec. 2.3 block Jacobi scaling,
 * Sec. 2.2 skeletonization) is one launch over the whole batch, and the host
 * plans and synchronizes once per level for all problems.  Problems with
 * fewer levels reach their root front earlier; it is eliminated as a cell of
 * that merged level.  The DOFs of the problems are numbered consecutively
 * (problem i's DOFs start at rhif_batch_info's dof_base[i]), and the handle
 * works on the concatenated vectors: rhif_apply and rhif_apply_noalloc apply
 * the block-diagonal F^{-1} of the batch, rhif_spmv the batch's A, rhif_pcg
 * runs PCG for every (problem, right-hand side) pair on concatenated vectors
 * (iters / relres then hold count x nrhs entries, problem-major), and
 * rhif_skeletons reports the units of all problems (DOFs in the concatenated
 * numbering).  rhif_estimate_es and rhif_autotune take single problems only.
 * A, g: HOST arrays of count entries (the CSR pointers are device pointers,
 * read during the call only).  Errors: those of rhif_factor; BAD_ARG for
 * count < 1, mixed dimensions or more than 2^31 - 1 DOFs in total. */
int rhif_factor_batch(int count, const rhif_csr* A, const rhif_grid* g, int leaf, double tol,
                      const rhif_opts* o, void* stream, rhif_handle** out);

/* Number of problems of a handle (1 for rhif_factor's) and, if dof_base is
 * not NULL, the first DOF of each problem in the concatenated numbering plus
 * the total (count + 1 HOST entries). */
int rhif_batch_info(const rhif_handle* F, int* count, int64_t* dof_base);

/* PCG for every problem of a merged batch handle with nrhs right-hand sides
 * each: f[i] and u[i] (HOST arrays of count DEVICE pointers) hold problem i's
 * N_i x nrhs right-hand sides and solutions (leading dimension N_i).  One
 * iteration advances every (problem, right-hand side) pair with the same
 * launches; each pair stops on its own relative residual (Sec. 4).  iters and
 * relres: HOST arrays of count * nrhs entries, problem-major.  Errors as
 * rhif_pcg; BAD_ARG for a handle of a single problem.  As in rhif_pcg, the
 * iterations run on the device as one CUDA graph whose conditional loop tests
 * every pair's convergence there (from the host while kernel timing is on). */
int rhif_pcg_batch(const rhif_handle* F, int nrhs, const double* const* f, double* const* u,
                   double rtol, int maxit, int* iters, double* relres, void* stream);

/* Autotuner of the scheduling options: one pass of coordinate descent over
 * big_front, big_frame, skel_cluster and (FP32 factors) tensor_cores, each
 * tried at its library default (0), forced on (1; skel_cluster: -1 and 4) and
 * forced off (-1), starting from `base` (NULL = defaults).  A configuration
 * costs the device time of rhif_factor (its event span, host planning gaps
 * included) plus `applies` times one F^{-1} application to one vector, the
 * smaller of two trials after one warm-up factorization; a change is kept
 * when it is at least 2% cheaper.  These options change only how the work is
 * split over CTAs (rounding order), never the factor's definition (Secs. 2-3),
 * so every candidate computes the same PHIF factor.  A is factored about 20
 * times.  *best receives the options (precision, precondition and
 * edge_skel_3d as in base), *best_ms (may be NULL) their cost.  Errors: those
 * of rhif_factor / rhif_apply; BAD_ARG for a NULL best or applies < 0. */
int rhif_autotune(const rhif_csr* A, const rhif_grid* g, int leaf, double tol, const rhif_opts* base,
                  int applies, void* stream, rhif_opts* best, double* best_ms);

/* PCG (as rhif_pcg) for `count` factored problems at once, each with nrhs
 * right-hand sides stored contiguously (f[i] and u[i] are N_i x nrhs with
 * leading dimension N_i), spread over the streams like rhif_factor_batched.
 * iters and relres are HOST arrays of count * nrhs entries (problem-major). */
int rhif_pcg_batched(int count, rhif_handle* const* F, int nrhs, const double* const* f,
                     double* const* u, double rtol, int maxit, int* iters, double* relres,
                     void* const* streams, int nstreams);

/* y = op(F) x for nrhs column vectors of length N stored with leading
 * dimensions ldx/ldy (>= N):
 *  - RHIF_SOLVE:  y = F^{-1} x (Eq. 3.2), the upward and downward sweeps;
 *  - RHIF_HALF:   y = G^{-1} x = B_L^{-1} R_{L-1}^T ... R_0^T x with F = G G^T
 *                 (Eq. 3.3), the upward sweep and the forward root solve;
 *  - RHIF_HALF_T: y = G^{-T} x, the backward root solve and the downward
 *                 sweep (so RHIF_HALF_T after RHIF_HALF is RHIF_SOLVE);
 *  - RHIF_MATVEC: y = F x (Eq. 3.1).  The stored factor keeps the explicit
 *                 inverses F^{-1} needs, so F x is the solution of
 *                 F^{-1} y = x by conjugate gradients preconditioned with A
 *                 (a few iterations: A F^{-1} is the operator PCG sees),
 *                 to ||x - F^{-1} y|| <= 1e-13 ||x|| for FP64 factors (1e-7
 *                 for FP32 ones) or the precision of the application; it
 *                 uses the handle's work space; single problems only.
 * x and y may alias only if ldx == ldy and x == y (not for RHIF_MATVEC).
 * Errors: BAD_ARG (unknown op, sizes, aliasing), CUDA. */
int rhif_apply(const rhif_handle* F, int op, int nrhs, const double* x, int64_t ldx,
               double* y, int64_t ldy, void* stream);

/* y = F^{-1} x like rhif_apply(F, RHIF_SOLVE, ...) but without allocating any
 * device memory.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate while they apply the preconditioner, for
 * instance an outer solver that has reserved all device memory up front, or
 * code that must not risk the device synchronization and mid-run allocation
 * failure that cudaMalloc can bring.  Scratch comes from a static device array
 * of 2^20 doubles (8 MiB) that every GPU loading the library holds until the
 * process exits; requests needing more (ub_len * nrhs, about the number of
 * boundary DOFs of one level times nrhs) are rejected with RHIF_ERR_BAD_ARG
 * before any work is queued.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) and should come before any stream
 * capture on that device.  All calls share the array: calls that overlap on
 * the GPU race and must be ordered by the caller.  Its launches are not
 * counted by the kernel instrumentation (rhif_kernel_stats). */
int rhif_apply_noalloc(const rhif_handle* F, int nrhs, const double* x, int64_t ldx,
                       double* y, int64_t ldy, void* stream);

/* y = A x with the stencil form of the A given to rhif_factor (FP64). */
int rhif_spmv(const rhif_handle* F, int nrhs, const double* x, int64_t ldx,
              double* y, int64_t ldy, void* stream);

/* PCG (Sec. 4) on A u = f with F^{-1} as the preconditioner, FP64 vectors,
 * x0 = 0, stopped when ||f - A u|| / ||f|| <= rtol (recursive residual) for
 * every right-hand side or after maxit iterations.  iters and relres are HOST
 * arrays of nrhs entries receiving the iteration count and the true relative
 * residual.  Returns NOT_CONVERGED if some system missed rtol.  The iterations
 * run on the device as one CUDA graph (captured once per u, nrhs, rtol and
 * maxit, on a private stream, and launched on `stream`) whose conditional
 * loop tests convergence on the device; the call returns after one wait for
 * the results.  While kernel timing is on (rhif_set_timing) the iterations
 * are issued from the host instead, one wait per iteration. */
int rhif_pcg(const rhif_handle* F, int nrhs, const double* f, int64_t ldf, double* u,
             int64_t ldu, double rtol, int maxit, int* iters, double* relres,
             void* stream);

/* Error estimate e_a = ||A - F||_2 / ||A||_2 (Sec. 4) by two power
 * iterations as in rhif_estimate_es: on (A - F)^2 from x0 (F x as in
 * rhif_apply with RHIF_MATVEC) and on A^2 from x1 (NULL: x0), each stopped
 * when two successive estimates differ by at most rel times the estimate or
 * after maxit products.  ea, iters (products of the first iteration): HOST
 * scalars.  Single problems only. */
int rhif_estimate_ea(const rhif_handle* F, const double* x0, const double* x1, int maxit,
                     double rel, double* ea, int* iters, void* stream);

/* Error estimate e_s = ||I - A F^{-1}||_2 (Sec. 4) by power iteration on
 * M^T M with M = I - A F^{-1}, M^T = I - F^{-1} A (A and F^{-1} symmetric):
 * v = x0 / ||x0||; repeat w = M^T M v, est = sqrt(||w||), v = w / ||w|| until
 * two successive estimates differ by at most rel * est or maxit products.
 * x0: DEVICE vector of N doubles (the start vector; the caller seeds it).
 * es, iters: HOST scalars receiving the estimate and the number of products.
 * Uses the handle's work space (no effect on the factor). */
int rhif_estimate_es(const rhif_handle* F, const double* x0, int maxit, double rel, double* es,
                     int* iters, void* stream);

/* C -= A B^T on the tensor cores (tcgen05, FP32 accumulation), the product
 * used for the dense Schur updates of large fronts (Sec. 2.1), exported so
 * that it can be checked on a device.  kind: RHIF_TC_TF32X3 (TF32 inputs split
 * into a high part and a remainder, three products: about FP32 accuracy),
 * RHIF_TC_TF32 (one TF32 product) or RHIF_TC_BF16 (inputs rounded to BF16).
 * A is M x K, B is N x K, C is M x N, all FP32 DEVICE arrays in column-major
 * order with leading dimensions lda, ldb, ldc; M, N >= 1, K >= 0.
 * RHIF_ERR_BAD_ARG for another kind or bad sizes, RHIF_ERR_TIMEOUT if a
 * bounded wait gave up. */
int rhif_tc_gemm_check(int kind, int M, int N, int K, const float* A, int64_t lda, const float* B,
                       int64_t ldb, float* C, int64_t ldc, void* stream);

/* Per-pixel gradient of a loss with respect to log a, given the state u and
 * the adjoint lam = A^{-1} dLoss/du:  grad_p = -a_p / 2^(d-1) *
 * sum over the grid edges e of pixel p of (lam_i - lam_j)(u_i - u_j)/h_e^2
 * (u = lam = 0 on boundary nodes).  Output grad has one value per pixel. */
int rhif_grad_logcoef(const rhif_grid* g, const double* a_pix, const double* u,
                      const double* lam, double* grad, void* stream);

typedef struct {
  int levels;             /* L */
  int64_t n;              /* N */
  int64_t root_size;      /* |S_L| */
  int64_t active[16];     /* |S_{l+1}| after level l, l < min(L,16) */
  int64_t factor_bytes;   /* device bytes held by the factor */
  double flops;           /* algorithmic flops of the factorization */
  double apply_bytes;     /* factor bytes streamed by one rhif_apply per rhs */
  int precision;
  int units;              /* skeletonized units, all levels */
  double factor_ms;       /* device time of the last rhif_factor */
  int fp64_leaves;        /* leaves of an FP32 factor re-eliminated in FP64 (leaf_fp64) */
  int64_t unit_dofs[16];  /* DOFs of the skeletonized units of level l (all phases) */
  int64_t skeletons[16];  /* of them kept as skeletons (sum of the ID ranks), l < min(L,16) */
} rhif_stats_t;

/* Copy statistics of a factor to host memory. */
int rhif_stats(const rhif_handle* F, rhif_stats_t* st);

/* Skeletonization record of one level/phase (phase 0 = edges in 2D, faces in
 * 3D; phase 1 = 3D edges).  Host outputs: *count units; for unit u, sizes[u]
 * DOFs and ranks[u] skeletons.  If gids != NULL it receives, unit after unit,
 * the sizes[u] DOF indices in pivot order (skeletons first); capacity is the
 * length of gids.  Call with gids == NULL first to learn the sizes. */
int rhif_skeletons(const rhif_handle* F, int level, int phase, int* count,
                   int* sizes, int* ranks, int64_t* gids, int64_t capacity);

/* Kernel instrumentation (process-wide).  Every kernel launch of the library
 * is counted per category; with timing on, CUDA events bracket each launch on
 * its stream and the elapsed times are summed when the statistics are read.
 * flops / bytes are the algorithmic work of the counted launches (see the
 * per-category work counts kept beside each launch in the library: factor
 * kernels count the flop formulas of Secs. 2.1-2.3, the application and vector
 * kernels the bytes of the factor blocks and vectors they stream). */
typedef struct {
  char name[32];
  int64_t launches;
  double total_ms;   /* 0 unless timing was on */
  double flops;
  double bytes;
} rhif_kernel_stat;

/* Turn per-launch CUDA-event timing on (1) or off (0); returns RHIF_OK. */
int rhif_set_timing(int on);
/* Zero every category's counters. */
int rhif_reset_kernel_stats(void);
/* Copy category `index` (0 <= index < rhif_kernel_stat_count()) to *out.
 * Synchronises the device once to resolve pending timing events. */
int rhif_kernel_stat_count(void);
int rhif_kernel_stats(int index, rhif_kernel_stat* out);

/* Release every device allocation of the handle (stream-ordered on the
 * stream of the factorization). */
void rhif_free(rhif_handle* F);

const char* rhif_error_string(int code);
const char* rhif_last_error_detail(void);

/* Host-only self-check of the level planner (Sec. 3.1, Fig. 3): builds the
 * plan of every level of a dim-D grid ns[0..dim-1] (leaf size `leaf`) with
 * seeded synthetic survivor flags (each DOF of a skeletonized group kept with
 * probability `keep`, splitmix64 stream from `seed`; edges too when
 * edge_skel_3d) and checks it against the definitions, recomputed from DOF
 * coordinates: bucket order by (code, index), cell interiors and segments,
 * the group-to-cell lists, every extend-add map entry (a surviving child
 * frame DOF lands on the same DOF of the parent front, a dropped one on -1),
 * and an identical rebuild from recycled storage.  No device work.  Writes
 * the number of levels checked to *levels_checked (may be null).  Returns
 * RHIF_OK, RHIF_ERR_BAD_ARG, or RHIF_ERR_CHECK with the first violation in
 * rhif_last_error_detail(). */
int rhif_plan_selfcheck(int dim, const int* ns, int leaf, double keep, uint64_t seed,
                        int edge_skel_3d, int64_t* levels_checked);

#ifdef __cplusplus
}
#endif
#endif /* RHIF_H */
