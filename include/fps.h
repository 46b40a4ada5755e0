/*
 * fps.h -- C ABI of the GB300 (sm_103a) spectral Poisson solver.
 *
 * The library solves the discretisation of Poisson's equation with homogeneous
 * Dirichlet conditions on [-1,1]^2 (and [-1,1]^3) in the normalised
 * ultraspherical basis C~^(3/2) of Fortunato & Townsend, "Fast Poisson solvers
 * for spectral methods" (arXiv 1710.11259):
 *
 *     square:  M X D^T + D X M^T = F                         (Sec. 3.2, eq. (3.6))
 *     cube:    (D_xx + D_yy + D_zz) vec(X) = vec(F)          (Sec. 5, eq. (5.2))
 *
 * with M the multiplication-by-(1-x^2) matrix of (3.7) and D = diag(-(j+1)(j+2)).
 * The solve is the ADI iteration of Algorithm 2 with the Zolotarev shifts of
 * Theorem 2.1 / eq. (2.4) and the iteration count of eq. (2.9), run on the
 * symmetrised equation (3.9).
 *
 * Conventions shared by every entry point
 *   - Matrices are row-major, FP64, contiguous.  X[i*n + j] pairs C~_i(y) with
 *     C~_j(x) (expansion (3.2)); F likewise.  Cube tensors are X[(i*n + j)*n + k].
 *   - Pointers may be device pointers (on the plan's device) or host pointers
 *     (pageable or pinned).  Device pointers: the call is asynchronous on the
 *     plan's stream and returns after enqueueing.  Host pointers: the library
 *     stages through its own device buffers and the call returns after the
 *     result has been copied back (it synchronises the plan's stream).
 *   - The caller owns F, X and gradient buffers; the plan owns everything else
 *     (shift table, per-shift Thomas factors, work arrays, CUDA graph).
 *   - F is never modified.  X must not overlap F.
 *   - Device buffers must be memory of the plan's device (of the current device for
 *     the plan-free calls) or managed memory; device memory of another device is
 *     rejected with INVALID_ARG.
 *   - Errors from argument checks are returned synchronously; errors from the
 *     device (a failed launch) are returned by the call that detects them.
 *     fps_last_error() gives a one-line message for the calling thread.
 *   - A plan is not thread-safe: use one plan per host thread.
 */
#ifndef FPS_H
#define FPS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fps_plan fps_plan;

/* Arithmetic of the ADI sweeps. */
typedef enum {
    FPS_FP64 = 0,        /* plain method: every sweep in FP64 */
    FPS_FP32_REFINE = 1  /* FP32 sweeps inside an FP64 iterative refinement of (3.9) */
} fps_precision;

/* Flag OR-ed into the precision argument of fps_plan_create: take the ADI shifts of
 * an FPS_FP64 square from a tight spectral interval of A~ (Sturm-count bisection,
 * fps_square_spectral_interval with tight != 0) instead of Lemma B.2's Gershgorin
 * interval; the cross-ratio of (2.9) shrinks, and so does J (133 -> 110 at n = 10^4,
 * tol 1e-13).  FPS_FP32_REFINE inner solves always use the tight interval. */
#define FPS_TIGHT_SPECTRUM 0x100

typedef enum {
    FPS_OK = 0,
    FPS_ERR_INVALID_ARG = -1,   /* bad size, tolerance, dimension, pointer */
    FPS_ERR_UNSUPPORTED = -2,   /* valid request the library does not implement */
    FPS_ERR_CUDA = -3,          /* a CUDA runtime call or launch failed */
    FPS_ERR_NOT_CONVERGED = -4, /* refinement missed its target; X holds the best iterate */
    FPS_ERR_NONFINITE = -5,     /* F (or an intermediate) holds NaN/Inf */
    FPS_ERR_TIMEOUT = -6        /* a bounded device-side wait gave up */
} fps_status;

/* Read-only facts about a plan. */
typedef struct {
    int64_t n;              /* problem size per dimension (largest n for a batch) */
    int dim;                /* 2 or 3 */
    int precision;          /* fps_precision */
    int nrhs;               /* right-hand sides per problem */
    int64_t batch;          /* problems in the plan (1 unless batched) */
    int J;                  /* ADI iterations of the FP64 solve, eq. (2.9) (cube: outer level) */
    int J_inner;            /* ADI iterations per refinement round (FP32_REFINE; cube: outer
                               level of a round) */
    int refine_rounds;      /* rounds used by the last FP32_REFINE solve */
    double last_residual;   /* max |R~| / max |F~| (cube: max |R| / max |G|) after the last
                               FP32_REFINE solve */
    double tol;             /* requested tolerance */
    int64_t device_bytes;   /* device memory owned by the plan */
    int64_t kernel_launches; /* kernels of this library launched by the last solve */
    int seg_len;            /* square plans: segment length of the partitioned sweeps (rows of a
                               column-pass tile, columns of a row-pass tile); FP32_REFINE: picked
                               by the autotuner unless FPS_AUTOTUNE=0 */
    int64_t inner_iterations; /* cube: inner (slice Stein) ADI iterations over full
                                 tensors in the last solve, all levels and rounds */
    int chain_mode;         /* square plans: load batching of the segment-coupling kernel
                               (1 short, 2 long batches; FP32_REFINE: picked by the autotuner
                               with seg_len, 0 = chosen by grid size when it did not run) */
} fps_plan_info_t;

/*
 * fps_plan_create -- plan the solve of one problem of size n (dim = 2: n x n;
 * dim = 3: n x n x n) for `nrhs` right-hand sides stored back to back.
 *   tol        relative accuracy eps of Theorem 2.1, 0 < tol < 1 (App. A requires it).
 *              FP64: the ADI error bound ||Y - Y_J||_2 <= tol ||Y||_2 of (2.9).
 *              FP32_REFINE: target of max |R~| / max |F~| for the refinement.
 *   precision  fps_precision, optionally | FPS_TIGHT_SPECTRUM (squares).
 *   stream     cudaStream_t (may be NULL for the legacy default stream); the
 *              plan's device is the current device at the time of the call.
 * The plan computes the spectral interval of Lemma B.2, J of (2.9), the shifts
 * of (2.4) on the host in FP64, uploads them and factors every shifted matrix
 * A~ - q_j I once (Thomas pivots, App. B even/odd decoupling).
 * Every shift list is validated on the host before any kernel runs (finite, inside
 * the spectral interval).  Environment: FPS_MAX_REFINE_ROUNDS caps the refinement
 * rounds of FP32_REFINE plans (default 8 for squares, 12 for cubes);
 * FPS_CUBE_SLICE=1 makes FP32 cube plans (n <= 256) run their inner level with the
 * slice-resident cluster kernel instead of the default whole-tensor line solves
 * (measured slower; kept as an option); FPS_INJECT_SHIFT_FAULT=nan|neg corrupts
 * the first shift before validation (host-side fault injection for tests).
 * Errors: INVALID_ARG (n < 1, dim not 2/3, tol outside (0,1), nrhs < 1, out NULL, a
 * shift list that fails validation), CUDA (allocation or launch failure).  *out is
 * NULL on error.
 */
int fps_plan_create(fps_plan **out, int64_t n, int dim, double tol, int precision, int nrhs, void *stream);

/*
 * fps_plan_create_rect -- plan Poisson's equation on the rectangle [x0, x0 + width] x
 * [y0, y0 + height] with homogeneous Dirichlet data (Sec. 3 on a rectangle).  The
 * affine map onto [-1,1]^2 multiplies u_xx by kx = (2/width)^2 and u_yy by
 * ky = (2/height)^2, so the discrete equation is kx M X D^T + ky D X M^T = F in the
 * mapped C~ coefficients (X[i*n + j] pairs C~_i(y) with C~_j(x)); in the variables of
 * (3.9) it is kx A~ Y + ky Y A~ = F~, a Sylvester equation whose two spectral
 * intervals differ, solved by Algorithm 2 with the general shifts of App. A.  Solve
 * with fps_poisson_square_solve (the adjoint is the same solve: the map stays
 * self-adjoint).  fps_plan_shifts returns the column-side shifts q_j.
 *   width, height  side lengths, positive and finite (only they matter, not x0, y0).
 *   others         as fps_plan_create for dim = 2 (precision may carry FPS_TIGHT_SPECTRUM).
 * Errors as fps_plan_create.
 */
int fps_plan_create_rect(fps_plan **out, int64_t n, double width, double height, double tol, int precision,
                         int nrhs, void *stream);

/*
 * fps_plan_create_batched -- plan `count` independent squares of sizes ns[0..count-1]
 * (each with its own J and shifts), each with `nrhs` right-hand sides.  Layout
 * of F and X: problem after problem, each problem's nrhs n_p x n_p matrices back
 * to back.  Errors as fps_plan_create, plus INVALID_ARG for count < 1 or ns NULL.
 */
int fps_plan_create_batched(fps_plan **out, const int64_t *ns, int64_t count, int nrhs, double tol, int precision,
                            void *stream);

/* Make later calls on this plan enqueue on `stream` (a cudaStream_t). */
int fps_plan_set_stream(fps_plan *plan, void *stream);

/*
 * fps_poisson_square_solve -- X = solution of (3.6) for F (per right-hand side,
 * per problem of a batch).  Algorithm 2 on A~ Y + Y A~ = F~ of (3.9), then
 * X = D_s Y D_s (the recovery consistent with the printed right-hand side of (3.9)).
 * Errors: INVALID_ARG (plan NULL or not dim 2, F/X NULL or overlapping, F/X device
 * memory of another device), NONFINITE (FP32_REFINE: F holds NaN/Inf), NOT_CONVERGED (FP32_REFINE missed tol),
 * CUDA.
 */
int fps_poisson_square_solve(fps_plan *plan, const double *F, double *X);

/*
 * fps_poisson_cube_solve -- X = solution of (5.2) on [-1,1]^3 by the nested ADI of
 * Sec. 5: outer split (T_01 + T_02) | T_12 of the symmetrised operator, middle
 * split of T_01 + T_02 + s into two halves, inner Stein equations
 * A~ Z A~ + c Z = R on every slice.  FPS_FP64: outer tolerance = the plan's tol,
 * middle and inner 1e-15, the paper's form of every level.  FPS_FP32_REFINE: the
 * nested ADI in FP32, every level in residual-propagating form, with level
 * tolerances (t, 1e-6, 1e-7), t in [1e-4, 1e-3] picked per plan for the fewest
 * outer iterations over the predicted rounds (a round reduces the residual by about
 * t/2), and every level's shifts on the Sturm-bisection
 * interval of A~ (Lemma B.2's interval for FPS_FP64), inside an FP64 defect
 * correction on the residual
 * R = G - (T_01 + T_02 + T_12) Y of the symmetrised equation (G = -F/sqrt(E_i E_j E_k))
 * until max |R| / max |G| <= tol (at most 12 rounds).  Plans: dim = 3, n <= 320.
 * X[(i*n + j)*n + k] pairs C~_i(x) C~_j(y) C~_k(z).  Host or device F and X.
 * Errors: INVALID_ARG (plan not dim 3, NULL/overlapping buffers, device memory of
 * another device), UNSUPPORTED
 * (n > 320 at plan creation), NONFINITE (FP32_REFINE: F holds NaN/Inf),
 * NOT_CONVERGED (FP32_REFINE missed tol; X holds the last iterate), CUDA.
 */
int fps_poisson_cube_solve(fps_plan *plan, const double *F, double *X);

/*
 * fps_poisson_adjoint -- dL/dF from dL/dX for the solve of this plan.  The
 * solve map F -> X is a rational function of the commuting symmetric operators
 * Y -> A~ Y and Y -> Y A~ wrapped by the diagonal scalings of (3.9), so it is
 * self-adjoint in the Frobenius inner product: the adjoint is the same ADI with
 * the same shifts applied to dL/dX.  Nothing from the forward solve is needed.
 * Errors as the corresponding solve.
 */
int fps_poisson_adjoint(fps_plan *plan, const double *dLdX, double *dLdF);

/* Fill *info.  Errors: INVALID_ARG. */
int fps_plan_info(const fps_plan *plan, fps_plan_info_t *info);

/*
 * fps_plan_shifts -- copy the plan's ADI shifts q_0..q_{J-1} (for the square,
 * p_j = -q_j) into q (capacity `cap`); returns the count written or a negative
 * status.  FPS_FP64: the shifts of the solve (Lemma B.2 interval, J of (2.9)).
 * FPS_FP32_REFINE: the shifts of the finest inner level (tight interval of A~,
 * tolerance 1e-7) of problem `problem` (0 unless batched).
 */
int fps_plan_shifts(const fps_plan *plan, int64_t problem, double *q, int cap);

/*
 * fps_plan_set_instrument -- on != 0: record CUDA events around every launch of
 * the plan's ADI pass kernels (the row pass and the column pass of every
 * iteration of Algorithm 2), inside the captured graphs, so that their duration
 * can be read after a solve without changing what runs.  Rebuilds the graphs.
 * Square plans only.  Errors: INVALID_ARG, UNSUPPORTED (cube plan), CUDA.
 */
int fps_plan_set_instrument(fps_plan *plan, int on);

/*
 * fps_plan_kernel_times -- for the last solve of an instrumented plan: number of
 * timed launches of the ADI pass kernels (*count, two per iteration), their summed
 * duration in ms (*total_ms) and the algorithmic bytes they move (*alg_bytes: per
 * element and iteration the residual-form ADI reads and writes six n x n words --
 * the row pass reads c and D and writes D and its result, the column pass reads
 * that result and writes c -- four in the first iteration, five in the second;
 * 8 bytes per FP64 and 4 per FP32 word; no padding, halo, segment-summary or
 * re-read traffic).  Synchronises the plan's stream.
 * Errors: INVALID_ARG (not instrumented), TIMEOUT (a bounded device wait gave up), CUDA.
 */
int fps_plan_kernel_times(fps_plan *plan, int *count, double *total_ms, double *alg_bytes);

/*
 * fps_plan_pass_times -- the summed durations (ms) of the row passes and of the
 * column passes of the last solve of an instrumented plan (their sum is the
 * *total_ms of fps_plan_kernel_times).  Errors as fps_plan_kernel_times.
 */
int fps_plan_pass_times(fps_plan *plan, double *row_ms, double *col_ms);

/*
 * fps_legendre_to_ctilde -- Legendre coefficients in (Sec. 3.4, Table 3.1 step 1):
 * F = C~^(3/2) coefficients of f = sum_{a,b < n} G[a*n + b] P_a(y) P_b(x), as used by
 * fps_poisson_square_solve.  With (2k+1) P_k = C^(3/2)_k - C^(3/2)_{k-2} the map is
 * banded: F = B G B^T, B[j][j] = 1/((2j+1) s_j), B[j][j+2] = -1/((2j+5) s_j),
 * C~_k = s_k C^(3/2)_k.  G and F: device pointers, n x n row-major, caller-owned,
 * not overlapping; asynchronous on `stream`.  Errors: INVALID_ARG (n < 1, NULL,
 * overlap, host memory or memory of a device other than the current one), CUDA.
 */
int fps_legendre_to_ctilde(int64_t n, const double *G, double *F, void *stream);

/*
 * fps_solution_to_legendre -- Legendre coefficients out (Sec. 3.4, Table 3.1 step 4):
 * U[i*(n+2) + k], i, k < n + 2, are the Legendre coefficients of the solution
 * u = (1-x^2)(1-y^2) sum_{i,j < n} X[i*n + j] C~_i(y) C~_j(x) of (3.1)-(3.2), i.e.
 * U = B^{-1} (M X M^T) B^{-T} with M of (3.7), computed as U = L X L^T with
 * L[j][j] = c_j, L[j+2][j] = -c_j, c_j = s_j (j+1)(j+2)/(2j+3).  X (n x n) and U
 * ((n+2) x (n+2)): device pointers, row-major, caller-owned, not overlapping;
 * asynchronous on `stream`.  Errors: INVALID_ARG (n < 1, NULL, overlap, host
 * memory or memory of a device other than the current one), CUDA.
 */
int fps_solution_to_legendre(int64_t n, const double *X, double *U, void *stream);

/*
 * fps_poisson_dirichlet_solve -- Poisson with nonhomogeneous Dirichlet data (Sec. 6.1)
 * on the plan's square or rectangle, in Legendre coefficients of the mapped
 * variables x, y in [-1, 1] (row index = degree in y, column index = degree in x):
 *   G   [nrhs][n][n]        f = sum G[a][b] P_a(y) P_b(x)
 *   bc  [nrhs][4][n+2]      the traces g_W = u(-1, y), g_E = u(1, y), g_S = u(x, -1),
 *                           g_N = u(x, 1), each sum_k bc[side][k] P_k(t)
 *   U   [nrhs][n+2][n+2]    u = sum U[i][j] P_i(y) P_j(x)  (output)
 * Sec. 6.1's four steps: (1) u_bc = the transfinite (Coons) interpolant of the traces
 * (each corner value the mean of the two traces meeting there, so u_bc takes every
 * trace exactly when the traces agree at the corners); (2) its Laplacian
 * kx u_bc,xx + ky u_bc,yy, exact in the n x n block for n >= 2; (3) the homogeneous
 * solve of the plan (Table 3.1 steps 1-4: F = B (G - lap u_bc) B^T, the ADI, the
 * output map); (4) U = that solution + u_bc.  The plan must be a single square
 * (fps_plan_create, dim 2) or rectangle (fps_plan_create_rect) plan, any precision,
 * its nrhs right-hand sides solved together.  Buffers: device memory of the plan's
 * device, caller-owned, U not overlapping G or bc; asynchronous on the plan's stream.
 * The plan allocates two n x n FP64 work arrays per right-hand side on the first
 * call and keeps them.  Errors: INVALID_ARG (NULL, host memory, overlap, batched or
 * cube plan), NOT_CONVERGED (FP32_REFINE plans: U then holds the last iterate's
 * solution), CUDA.
 */
int fps_poisson_dirichlet_solve(fps_plan *plan, const double *G, const double *bc, double *U);

/*
 * fps_poisson_dirichlet_adjoint -- gradients of a loss L(U) through
 * fps_poisson_dirichlet_solve: given dLdU [nrhs][n+2][n+2] it writes dLdG [nrhs][n][n]
 * and dLdbc [nrhs][4][n+2], the transpose of the linear map (G, bc) -> U applied to
 * dLdU: the transposed output map, the same ADI solve (the solve map is
 * self-adjoint), the transposed input map, and for the traces the transposed lifting
 * minus the transposed Laplacian of the lifting applied to dLdG.  Same plan, buffer
 * and error rules as the solve; the three buffers must not overlap.
 */
int fps_poisson_dirichlet_adjoint(fps_plan *plan, const double *dLdU, double *dLdG, double *dLdbc);

/*
 * fps_plan_create_cylinder -- the Fourier modes k = kmin .. kmax (2 <= kmin) of
 * Poisson's equation on the cylinder after the doubling-up of Sec. 4.1 (Case 1):
 * for each mode, u_k(r, z) = r^2 (1 - r^2)(1 - z^2) w_k(r, z) with
 * w_k = sum_{i,j < n} Y[i][j] C~_i(r) C~_j(z) solving
 *     P Y M^T + Q Y D = F,   P = L1 - k^2 M,  Q = M_{r^2} M,
 * L1 the matrix of r^2(1-r^2) d^2/dr^2 + (5-9r^2) r d/dr + 4(1-4r^2) (equal to
 * M_{r^2} D + 5 M_r M D_1 + 14 M - 10 I), M of (3.7), D = diag(-(j+1)(j+2)); F the
 * C~ x C~ coefficients of the mode's right-hand side f_k(r, z) (row index = degree in
 * r).  The ADI of Algorithm 2 runs on A Y - Y B = P^{-1} F D^{-1}, A = P^{-1} Q,
 * B = -M D^{-1}, multiplied through by P so that only banded solves and products
 * remain; shifts (2.4) per mode from an interval of sigma(A_k) found by power
 * iteration (widened by 3 %) and the tight interval of sigma(B); J of (2.9) per mode.
 * FP64.  n >= 4, nrhs right-hand sides per mode (e.g. the real and imaginary parts
 * of f_k and f_{-k}).  The line kernels hold 32 whole lines per CTA in shared memory
 * (about 352 n bytes), so n is bounded by the device's per-CTA limit: n <= 660 on
 * GB300 (227 KB).  Errors: INVALID_ARG, UNSUPPORTED (n above that bound or above
 * 4096, an interval or a pivot that cannot be formed), CUDA.
 */
int fps_plan_create_cylinder(fps_plan **out, int64_t n, int64_t kmin, int64_t kmax, double tol, int nrhs,
                             void *stream);

/*
 * fps_poisson_cylinder_solve -- Y for every (mode, right-hand side) of a cylinder plan.
 * F, Y: device pointers of the plan's device, [kmax - kmin + 1][nrhs][n][n] row-major,
 * caller-owned, not overlapping; asynchronous on the plan's stream.  Errors:
 * INVALID_ARG (not a cylinder plan, NULL, overlap, host memory or memory of another
 * device), CUDA.
 */
int fps_poisson_cylinder_solve(fps_plan *plan, const double *F, double *Y);

/*
 * fps_cylinder_mode_interval -- host helper: the interval [*a, *b] (a < b < 0) the
 * cylinder plan uses for sigma(A_k), A_k = P^{-1} Q of size n.  Errors: INVALID_ARG
 * (n outside [4, 4096], k < 2, NULL), UNSUPPORTED.
 */
int fps_cylinder_mode_interval(int64_t n, int64_t k, double *a, double *b);

/*
 * fps_cylinder_operators -- host helper: L1 and Q (n x n, row-major, caller-owned) of
 * the cylinder modes, from the closed forms the plans use (k is not used: P = L1 -
 * k^2 M).  Errors: INVALID_ARG.
 */
int fps_cylinder_operators(int64_t n, int64_t k, double *L1, double *Q);

/*
 * fps_poisson_square_solve_noalloc -- the FP64 square solve of fps_poisson_square_solve
 * (same shifts, iteration count and kernels) for n <= 256, without allocating
 * anything.  The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory when they solve (a caching allocator that owns the
 * device memory, hosts that forbid allocation after start-up, code that must avoid
 * the synchronisation cudaMalloc/cudaFree can cause).  No plan is needed.
 *   n       1 <= n <= 256;  tol in (0, 1) with J of (2.9) at most 256.
 *   F, X    device pointers (the caller allocates them), n x n row-major FP64,
 *           not overlapping; F is not modified.
 *   stream  cudaStream_t the work is enqueued on (asynchronous; NULL = legacy stream).
 * Work arrays live in one fixed 4 MiB device array inside the library that every
 * GPU loading the library holds until the process exits.  The first call on a
 * device looks its address up (cudaGetSymbolAddress) with that device current:
 * make that first call before any stream capture.  All calls on a device share the
 * array, which keeps the last call's contents (each call rewrites everything it
 * reads); calls that overlap on the GPU race on it, so order them on one stream.
 * Nothing is copied from host memory (the bands of A~ are computed on the device,
 * the shifts travel as a kernel argument).
 * Errors: INVALID_ARG (n or tol out of range, NULL/overlapping F or X, F or X not
 * device memory of the current device), CUDA.  fps_last_error() then returns a
 * fixed message (a string literal: reporting the error allocates nothing).
 */
int fps_poisson_square_solve_noalloc(int64_t n, double tol, const double *F, double *X, void *stream);

/* Release every resource of the plan (synchronises its stream).  NULL is a no-op. */
void fps_plan_destroy(fps_plan *plan);

/* Static one-line description of a status code. */
const char *fps_status_string(int status);

/* Message describing the most recent error on the calling thread ("" if none). */
const char *fps_last_error(void);

/* ---------------- host-only helpers (no GPU needed) ---------------- */

/*
 * fps_zolotarev_shifts -- ADI shifts of Theorem 2.1 for A X - X B = F with
 * sigma(A) in [a,b], sigma(B) in [c,d], a < b < c < d, 0 < tol < 1.
 * J <= 0 selects J from (2.9).  Writes *J_out; if p and q are non-NULL they
 * receive J values each (capacity `cap`).  Computed in FP64 on the host.
 * Errors: INVALID_ARG (interval order, tol, capacity too small).
 */
int fps_zolotarev_shifts(double a, double b, double c, double d, double tol, int J, int *J_out, double *p, double *q,
                         int cap);

/*
 * fps_square_bands -- the symmetric A~ of (3.9) for size n: diagonal d[0..n-1]
 * and coupling e[j] = A~[j][j+2] for j < n-2.  Host FP64.  Errors: INVALID_ARG.
 */
int fps_square_bands(int64_t n, double *d, double *e);

/*
 * fps_square_spectral_interval -- bounds sigma(A~) in [-hi, -lo] for size n.
 * tight = 0: Lemma B.2, lo = 1/(30 n^4), hi = 1 (the interval the FP64 solve and its
 * shift list use).  tight != 0: Sturm-count bisection on the even and odd
 * tridiagonals of A~ (App. B), lo = |lambda_max|/2 and hi = 1.01 |lambda_min| (the
 * interval of the FP32 inner solves, whose result is checked against the exact
 * solution rather than iterate by iterate).  Host FP64.  Errors: INVALID_ARG.
 */
int fps_square_spectral_interval(int64_t n, int tight, double *lo, double *hi);

/*
 * fps_probe_fma_rate -- measure the current device's fused multiply-add rate:
 * FP64 FMAs per second (precision = FPS_FP64) or FP32 ones (FPS_FP32_REFINE), from a
 * ~100 ms kernel of independent FMA chains timed with CUDA events.  Instrumentation
 * with no counterpart in the paper: it is the peak that the FP64 sweeps, bound by
 * GB300's FP64 rate rather than by HBM, are reported against.  Synchronous.
 * Errors: INVALID_ARG (NULL output, unknown precision), CUDA.
 */
int fps_probe_fma_rate(int precision, double *fma_per_s);

/* Build identification (compute capability the kernels were built for, e.g. 103). */
int fps_build_arch(void);

#ifdef __cplusplus
}
#endif

#endif /* FPS_H */
