/*
 * sg.h -- C ABI of the GB300 stochastic Galerkin (SG) solver.
 *
 * Method: Zheng, Lin and Xu, "Block Triangular Preconditioning for Stochastic
 * Galerkin Method" (arXiv 1304.1755).  Problem (Sec. 2, Eq. model-problem):
 *   -div(a(x, xi) grad u) = f on the unit square, u = 0 on the boundary,
 *   a = abar(x) + sum_{k=1}^M sqrt(lambda_k) b_k(x) xi_k   (Eq. truncated-KLE),
 * discretised by Q1 finite elements on a uniform (n x n)-vertex grid (or, with
 * elements = SG_P1, by the paper's linear triangles on the same grid, Sec. 6) and a
 * total-degree-p orthonormal polynomial chaos (Legendre or Hermite).  The
 * Galerkin matrix is A = sum_{k=0}^M G_k (x) K_k (Eq. tensor-product); it is
 * never assembled.
 *
 * Data layout of every SG vector (X, Y, R, Z, F, U):  PC-major,
 *   V[i * N_x + s],  i = 0..P-1 (PC index, degree-graded), s = 0..N_x-1,
 *   N_x = (n-2)^2 interior nodes, s = (vx-1) + (vy-1)(n-2) for vertex (vx, vy)
 *   (x1 fastest).  P = (M+p)!/(M! p!).
 * Element types: SG_F64 = double, SG_F32 = float, SG_BF16 = bfloat16 (raw
 * uint16 bit pattern of the upper half of an IEEE float).
 *
 * Ownership: the caller owns every buffer passed in; the handle owns the
 * operator data and all workspace (device memory, allocated at setup and on
 * first use of a precision).  Calls are ordered on the handle's CUDA stream;
 * functions that return host-visible results (sg_solve, sg_objective,
 * sg_adjoint_gradients) synchronise that stream before returning.
 * A handle is not thread-safe; distinct handles are independent.
 *
 * Errors: every function returns an sg_status (0 = success, negative =
 * failure); no exception crosses the ABI.  sg_last_error() gives a message.
 * After SG_E_CUDA the handle should be destroyed.
 */
#ifndef SG_GB300_H
#define SG_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sg_ctx* sg_handle;

typedef enum {
  SG_OK = 0,
  SG_E_ARG = -1,        /* invalid argument (sizes, pointers, options) */
  SG_E_ALLOC = -2,      /* device or host allocation failed */
  SG_E_CUDA = -3,       /* a CUDA runtime call failed */
  SG_E_NOCONV = -4,     /* solver hit maxit before the tolerance */
  SG_E_BREAKDOWN = -5,  /* Krylov breakdown (zero or non-positive pivot) */
  SG_E_NONFINITE = -6,  /* NaN or Inf met in a residual or inner product */
  SG_E_TIMEOUT = -7,    /* a bounded device-side wait gave up */
  SG_E_STATE = -8       /* call not valid in the handle's current state */
} sg_status;

/* SG_DF64: "double-float" storage of an N-element vector as 2N floats, the
 * leading parts hi[0..N) followed by the trailing parts lo[N..2N), value
 * hi + lo (about 48 significant bits).  It is the internal FP64-class format
 * of the fast solver mode (GB300 runs FP64 arithmetic at 1/68 of its FP32
 * rate); sg_apply accepts it for X and Y. */
/* SG_BF16Z (preconditioners and sg_solve's pc_prec only): the V-cycle levels and the
 * stage right-hand sides of the sweeps are stored in BF16 (FP32 arithmetic), the
 * preconditioned vectors Z = B^{-1} R the call returns are FP32.  Keeping the output
 * in FP32 avoids the BF16 rounding of the flexible basis z_j, which costs FGMRES
 * extra iterations, while the multigrid traffic stays at BF16 width. */
typedef enum { SG_F64 = 0, SG_F32 = 1, SG_BF16 = 2, SG_DF64 = 3, SG_BF16Z = 4 } sg_prec;
/* Arithmetic of the outer Krylov solver (the preconditioner's own arithmetic is set by pc_prec):
 *   SG_ARITH_F64: IEEE FP64 throughout -- Arnoldi basis, outer operator A z_j,
 *     Gram-Schmidt, Givens/least-squares update and true residual.
 *   SG_ARITH_F64_DFOP: as SG_ARITH_F64 (FP64 basis, FP64 Gram-Schmidt, FP64 Givens
 *     update on the host, IEEE FP64 true residual at every restart and at the end),
 *     except that the outer operator w = A z_j of each Arnoldi step is evaluated in
 *     double-float arithmetic (FP32 pairs with error-free transformations, about 48
 *     significant bits; the FP32/BF16 z_j are exact in it) and w is rounded to FP64 on
 *     the store.  GMRES/FGMRES with an SG_F32, SG_BF16 or SG_BF16Z preconditioner.
 *   SG_ARITH_DF64: the Arnoldi basis, the outer operator and the Gram-Schmidt sums
 *     in double-float (48-bit significand, FP32 exponent range); the Givens update on
 *     the host in FP64; every true residual (restart and final) in IEEE FP64.
 *     FGMRES with an SG_F32, SG_BF16 or SG_BF16Z preconditioner. */
typedef enum { SG_ARITH_F64 = 0, SG_ARITH_DF64 = 1, SG_ARITH_F64_DFOP = 2 } sg_arith;
typedef enum { SG_LEGENDRE = 0, SG_HERMITE = 1 } sg_family;
/* Spatial discretisation.  SG_Q1: bilinear elements on the square cells (the configurations' form).
 * SG_P1: the paper's own discretisation (Sec. 6): every cell cut by its SW-NE diagonal into a lower-
 * right and an upper-left right triangle, linear elements, the coefficient constant per triangle, so
 * each K_k is a 5-point stencil with edge weights; its V-cycle smooths with point Gauss-Seidel
 * (forward sweeps before, backward after the coarse correction, nu1 / nu2 of them; lexicographic or
 * red-black order, sg_gs_order),
 * prolongs by linear interpolation on the nested triangulations and restricts by its transpose.  SG_P1
 * handles take per-triangle coefficients, need a mean coefficient of exactly 1 (every coarse operator
 * is then the 5-point Laplacian) and compute in FP64 only: operators and preconditioners with
 * SG_F64, solves with pc_prec = SG_F64 and arith = SG_ARITH_F64; the allocation-free V-cycle, the
 * tile autotuner and the adjoint gradients are Q1-only. */
typedef enum { SG_Q1 = 0, SG_P1 = 1 } sg_elements;
/* Point Gauss-Seidel order of the SG_P1 V-cycle.  SG_GS_LEX: lexicographic (x fastest); the forward
 * sweep updates a node after its west and south neighbours, the backward sweep in the reverse order.
 * SG_GS_RB: red-black, colour (x + y) mod 2; the forward sweep updates colour 0 then colour 1, the
 * backward sweep colour 1 then colour 0 (both forms make the cycle a symmetric operator). */
typedef enum { SG_GS_LEX = 0, SG_GS_RB = 1 } sg_gs_order;
/* SG_BGS: the stationary block Gauss-Seidel iteration U += B_T^{-1}(F - A U) (Sec. 4.2). */
typedef enum { SG_GMRES = 0, SG_FGMRES = 1, SG_GPCG = 2, SG_PCG = 3, SG_BGS = 4 } sg_method;
/* SG_PC_BLOCKSYM: B_S = B_T diag(A)^{-1} B_T^T, the symmetric block Gauss-Seidel
 * preconditioner of Sec. 4.2 (lower sweep, the exact diagonal blocks K_0, upper sweep).
 * SG_PC_BLOCKTRI_EXACT: the 2 x 2 block-triangular form of Sec. 4.2 / Theorem 1,
 * B = [A_hat 0; W D] with A_hat the Galerkin matrix of total degree p-1 solved by an inner
 * FGMRES (right-preconditioned by the flat B_T of A_hat, to inner_tol) and the degree-p
 * diagonal blocks D = I (x) K_0 by one V-cycle each (see sg_precond_blocktri_exact).
 * With FGMRES and pc_prec = SG_F64 only; an analysis form, each application costs a solve.
 * SG_PC_BLOCKSYM_REC: the symmetric 2 x 2 form of Sec. 4.2, B_S = [A_hat 0; W D] diag(A_hat, D)^{-1}
 * [A_hat W^T; 0 D], applied recursively over the degree levels (A_hat^{-1} replaced by the same
 * preconditioner one degree lower, down to the mean block; D = I (x) K_0 by one V-cycle per block);
 * symmetric, for PCG; pc_prec = SG_F64 only (see sg_precond_blocksym_rec). */
typedef enum {
  SG_PC_NONE = 0,
  SG_PC_BLOCKTRI = 1,
  SG_PC_BLOCKDIAG = 2,
  SG_PC_BLOCKSYM = 3,
  SG_PC_BLOCKTRI_EXACT = 4,
  SG_PC_BLOCKSYM_REC = 5
} sg_pc;

/* One SG problem (Sec. 2-3).  coef is a HOST array of (M+1) rows of (n-1)^2
 * per-cell values, cell e = cx + cy (n-1): row 0 is the mean coefficient
 * abar_e (defines K_0, Eq. def-stiffness), row k >= 1 is
 * c_k(e) = sqrt(lambda_k) b_k(x_e) (times sigma), defining K_k.  For elements =
 * SG_P1 each row holds 2 (n-1)^2 per-triangle values instead, 2e the lower-right and
 * 2e + 1 the upper-left triangle of cell e (see sg_kl_coef_p1).  The handle
 * copies it.  n = 2^L + 1 with 3 <= n <= 4097; 0 <= M <= 16; 0 <= p <= 10;
 * P <= 4096.  nu1, nu2: pre/post smoothing steps of the V-cycle (damped Jacobi
 * for SG_Q1, point Gauss-Seidel sweeps for SG_P1; 0 selects 1; at most 4); omega:
 * Jacobi weight (0 selects 8/9; unused by SG_P1).  elements: sg_elements (0 = SG_Q1).
 * gs_order: sg_gs_order of the SG_P1 smoother (ignored by SG_Q1). */
typedef struct {
  int n;
  int M;
  int p;
  int family;
  const double* coef;
  int nu1;
  int nu2;
  double omega;
  int elements;
  int gs_order;
} sg_problem;

/* Solver options (Sec. 4.2, 6).  method: GMRES (right preconditioned) or
 * FGMRES (flexible: stores z_j = B^{-1} v_j in pc_prec) or GPCG[1] or PCG or the
 * stationary block Gauss-Seidel iteration.  precond: sg_pc (B_T, B_D, B_S, the exact
 * 2 x 2 B_T, the recursive 2 x 2 B_S, or none).  restart: Krylov
 * dimension m of (F)GMRES(m) (1..32).  maxit: maximum preconditioner
 * applications.  tol: stop when ||F - A U||_2 / ||F||_2 <= tol (true residual,
 * recomputed in FP64 at every restart and at the end).  pc_prec: precision of
 * the preconditioner (V-cycle and triangular sweep: SG_F64, SG_F32, SG_BF16 or
 * SG_BF16Z; z_j is stored in FP32 for SG_BF16Z); the coarsest-grid solve is FP64 in
 * every mode.  The arithmetic of the outer Krylov vectors, operator and
 * orthogonalisation is chosen by arith (sg_arith above); the Givens rotations and
 * the true residual are FP64 in every mode.  transpose: solve A^T U = F preconditioned by B^T (the
 * adjoint solve; B_T^T is the upper block-triangular sweep).  x0_given: U holds
 * an initial guess (else U = 0 is used).  reorth: 0 classical Gram-Schmidt,
 * 1 classical Gram-Schmidt with a second pass when the norm drops by more than
 * 1/sqrt(2) (selective reorthogonalisation).  arith: sg_arith.  inner_tol, inner_restart:
 * tolerance (0 selects 1e-12) and restart (0 selects 30) of the inner solves of
 * SG_PC_BLOCKTRI_EXACT; ignored by the other preconditioners. */
typedef struct {
  int method;
  int precond;
  int restart;
  int maxit;
  double tol;
  int pc_prec;
  int transpose;
  int x0_given;
  int reorth;
  int arith;
  double inner_tol;
  int inner_restart;
} sg_solve_opts;

/* Filled by sg_solve. iters = preconditioner applications (Arnoldi steps);
 * relres_est = the recurrence's residual estimate; relres_true = recomputed
 * ||F - A U|| / ||F|| in FP64; times are wall clock (ms) measured with CUDA
 * events on the handle's stream. */
typedef struct {
  int iters;
  int restarts;
  int status;
  double relres_est;
  double relres_true;
  double t_total_ms;
  int n_apply;
  int n_precond;
} sg_solve_info;

/* Host helper (Sec. 2.1, Eqs. truncated-KLE and exponential-covariance):
 * fills coef_out ((M+1) x (n-1)^2, host) with row 0 = abar (or 1 where abar is
 * NULL) and row k = sigma sqrt(lambda_k) b_k(cell centre) for the separable
 * covariance exp(-|x1-y1|/L - |x2-y2|/L), L = corr_len, modes sorted by
 * decreasing lambda (ties: lower x1-mode index first).  lambda_out (host, M
 * values) may be NULL.  Pure host computation, no device use. */
int sg_kl_coef(int n, int M, double sigma, double corr_len, const double* abar,
               double* coef_out, double* lambda_out);

/* Host helper for SG_P1 handles (the paper's discretisation, Sec. 6): coef_out ((M+1) x 2 (n-1)^2,
 * host) with row 0 = 1 and row k = sigma sqrt(lambda_k) b_k at the centroids of the two triangles of
 * every cell (lower-right at (2/3, 1/3), upper-left at (1/3, 2/3) of the cell), the same modes as
 * sg_kl_coef.  lambda_out may be NULL.  Pure host computation. */
int sg_kl_coef_p1(int n, int M, double sigma, double corr_len, double* coef_out, double* lambda_out);

/* Host helper, coercivity check of a coefficient set (Sec. 2.1: the paper's
 * assumption that a stays above a positive constant, and its remark that the
 * truncated expansion can violate it): *amin_out = min over the (n-1)^2 cells of
 * min_{|xi_k| <= xi_max} a(x_e, xi) = coef[0][e] - xi_max sum_{k>=1} |coef[k][e]|
 * (a is linear in xi, so the minimum is at a corner of the box).  xi_max = sqrt(3)
 * is the support of the Legendre chaos variables; Hermite variables are unbounded,
 * so there xi_max is a reference radius chosen by the caller.  coef as in sg_problem
 * (host, (M+1) x (n-1)^2).  Pure host computation, no device use. */
int sg_min_coef(int n, int M, const double* coef, double xi_max, double* amin_out);

/* Build a handle: uploads coefficients, basis tables and the multigrid
 * hierarchy (Galerkin coarse stencils when abar is not constant 1).  stream is
 * a cudaStream_t (NULL = legacy default stream). */
int sg_setup(const sg_problem* prob, void* stream, sg_handle* out);
void sg_destroy(sg_handle h);
int sg_set_stream(sg_handle h, void* stream);
const char* sg_last_error(sg_handle h);   /* h may be NULL: last setup error */

/* Sizes: N_x, P, number of multigrid levels (each may be NULL). */
int sg_sizes(sg_handle h, int* Nx, int* P, int* nlevels);
/* Multi-indices of the PC basis (host array P x M, row i = alpha_i),
 * degree-graded order (Sec. 3.3). */
int sg_basis(sg_handle h, int* alpha);

/* Load vector of the SG system (Eq. tensor-product's right-hand side): f is
 * deterministic, so only the mean PC block is nonzero, F = e_0 (x) F_0, with the
 * lumped load F_0[s] = h^2 f_s (h = 1/(n-1); for Q1 exact with constant f, for SG_P1 the lumped
 * mass of the six triangles around a vertex).  f_nodes: the
 * N_x interior nodal values of f (device, FP64), or NULL for f = 1.  F: device,
 * FP64, P * N_x values, fully overwritten (the blocks i >= 1 are set to zero).
 * Stream-ordered on the handle's stream; returns before the kernel finishes. */
int sg_rhs(sg_handle h, const double* f_nodes, double* F);

/* Y = A X (Eq. tensor-product), device X, Y in precision prec; arithmetic in
 * FP64 for SG_F64, double-float for SG_DF64, FP32 otherwise. */
int sg_apply(sg_handle h, const void* X, void* Y, int prec);
/* R = F - A U in FP64 (device F, U, R; R may alias F). */
int sg_residual(sg_handle h, const double* F, const double* U, double* R);

/* Z = B_T^{-1} R (Sec. 4.2): block forward substitution over the degree
 * levels q = 0..p, each diagonal block K_0 approximated by one V-cycle; with
 * transpose != 0, Z = B_T^{-T} R (backward over q = p..0).  R is FP64 (device),
 * Z is in precision prec (device); intermediate storage in prec. */
int sg_precond_blocktri(sg_handle h, const double* R, void* Z, int prec, int transpose);
/* Z = B_D^{-1} R (Sec. 4.1): one V-cycle on every PC block. */
int sg_precond_blockdiag(sg_handle h, const double* R, void* Z, int prec);
/* Z = B^{-1} R for the 2 x 2 block-triangular preconditioner of Sec. 4.2 whose lower-degree block
 * is the exact A_hat (Theorem 1's form; Eq. hierarchical_structure splits A_p into A_hat = A_{p-1},
 * the coupling W and the degree-p diagonal D = I (x) K_0):
 *   Z_low = A_hat^{-1} R_low,  Z_p = D^{-1}(R_p - W Z_low)           (transpose = 0)
 *   Z_p = D^{-T} R_p,          Z_low = A_hat^{-T}(R_low - W^T Z_p)  (transpose != 0).
 * A_hat^{-1} is an inner FGMRES(30) solve to a relative residual of inner_tol (0 selects 1e-12),
 * right-preconditioned by the flat B_T of A_hat in FP64, on a degree-(p-1) handle the first call
 * creates and the handle keeps; D^{-1} is one FP64 V-cycle per block.  R, Z: device FP64,
 * P * N_x values (Z must not alias R).  For p = 0 (no lower block) this is one V-cycle.
 * Synchronises the handle's stream (the inner solves do); returns the inner solve's status
 * (SG_E_NOCONV when it reached its iteration limit, Z then holds its last iterate). */
int sg_precond_blocktri_exact(sg_handle h, const double* R, double* Z, int transpose, double inner_tol);
/* Z = B_S^{-1} R (Sec. 4.2): lower sweep, multiplication by the diagonal blocks K_0
 * (exact), upper sweep; symmetric positive definite, for PCG.  R FP64, Z in prec. */
int sg_precond_blocksym(sg_handle h, const double* R, void* Z, int prec);
/* Z = B_S^{-1} R with the 2 x 2 symmetric form of Sec. 4.2 applied recursively over the degree levels:
 * for the top degree q, y_low = B_{q-1}^{-1} R_low, y_q = D^{-1} (R_q - W y_low),
 * z_low = B_{q-1}^{-1} (R_low - W^T y_q), Z = [z_low; y_q], with B_0^{-1} one V-cycle on the mean block
 * and D^{-1} one V-cycle per block of degree q (W: the couplings of degree q to degree q - 1).  The
 * degree-q' blocks are cycled 2^(p - q') times, so an application costs about twice a B_T sweep at
 * p = 4.  R, Z: device FP64, P * N_x values (Z must not alias R).  Allocates a workspace of about p
 * SG vectors on first use.  Stream-ordered; returns before the kernels finish. */
int sg_precond_blocksym_rec(sg_handle h, const double* R, double* Z);
/* One V(nu1,nu2) cycle on K_0 from a zero guess for nblocks stacked blocks of
 * N_x values: B FP64 (device), X in prec (device). */
int sg_vcycle(sg_handle h, const double* B, void* X, int nblocks, int prec);
/* sg_vcycle without any device allocation (the paper has no counterpart: this is a
 * library-usage variant of the V-cycle of Sec. 4.1).  Same arguments and result as
 * sg_vcycle for prec = SG_F64, SG_F32 or SG_BF16 (other precisions return SG_E_ARG),
 * but the coarse-level buffers come from one fixed 32 MiB array compiled
 * into the library instead of the handle's workspace, which sg_vcycle allocates on
 * its first call.  It is meant for callers that must not allocate: code running
 * under a caching allocator that already holds the device's free memory, or inside
 * latency-bound loops where cudaMalloc's implicit device synchronisation is not
 * acceptable.  Needs 2 * sum_{l=1..lc} round_up(s * nblocks * N_l, 256) bytes (s =
 * bytes per value of prec, N_l the interior nodes of level l, lc the last level
 * handled by the level kernels; 0 for n <= 33); a request above 32 MiB returns
 * SG_E_ARG with the required size in sg_last_error and launches nothing.  The first
 * call on each device (made with that device current) looks up the array's device
 * address; make that first call before capturing a stream into a CUDA graph.  All
 * calls in the process share the one array per device and it keeps the last call's
 * contents (nothing in it needs clearing: a call writes every value before reading
 * it), so calls that overlap in time, from any handle or stream, race and give
 * wrong results: serialise them. */
int sg_vcycle_static(sg_handle h, const double* B, void* X, int nblocks, int prec);

/* Solve A U = F (or A^T U = F).  F, U: FP64, host or device pointers (host
 * buffers are staged through device memory inside the call; page-locked ones copy
 * fastest, and for GMRES/FGMRES a page-locked U receives each restart's iterate on a
 * side stream while its true residual is checked, so the converged solution is already
 * on the host when the check confirms it).  info may be NULL.  Returns SG_E_NOCONV if
 * maxit is reached (U then holds the last iterate).  U is complete when the call
 * returns. */
int sg_solve(sg_handle h, const double* F, double* U, const sg_solve_opts* opts, sg_solve_info* info);

/* Solve nsys independent systems, each with its own handle (any mix of grids, M and p;
 * the batched form of the method's solve, Sec. 4.2 / 6, for many problems at once).
 * hs[s], F[s], U[s] as in sg_solve (device pointers); the same opts for every system.
 * The handles must be distinct (a handle's workspace serves one solve at a time); a repeated
 * handle is rejected with SG_E_ARG before any work starts.
 * nstreams (1..64) worker threads each drive one CUDA stream created for the call and
 * take the systems largest first; each handle's own stream is restored afterwards.
 * infos (may be NULL) receives one sg_solve_info per system, with status set to that
 * system's sg_solve result.  Returns SG_OK or the first failing system's status.
 * Handles must be distinct and not used by other calls while the batch runs. */
int sg_solve_batch(sg_handle* hs, const double* const* F, double* const* U, int nsys, const sg_solve_opts* opts,
                   sg_solve_info* infos, int nstreams);

/* The same batch as sg_solve_batch, solved in one CUDA graph (the batched form of the method's solve,
 * Sec. 4.2 / 6): every system's FGMRES restart cycle, with its Arnoldi scalars (Gram-Schmidt
 * coefficients, Hessenberg column, Givens rotations, convergence test, back substitution) computed by
 * one-thread kernels on the device and every further step behind a conditional graph node that the
 * previous step opens, is a chain of nodes; the chains of all systems sit side by side in one graph,
 * and one launch of it runs one restart cycle of the whole batch.  The call builds and instantiates the
 * graph, launches it until no system is running (normally once or twice), and reads each system's
 * outcome once per launch.  FGMRES with an FP64 basis only (arith SG_ARITH_F64, or SG_ARITH_F64_DFOP
 * with an SG_F32, SG_BF16 or SG_BF16Z preconditioner), restart 1..32, x0_given = 0, reorth = 0; F[s] and
 * U[s] device FP64; handles distinct, on the current device, and not used by other calls meanwhile (each
 * handle's stream is restored afterwards).  infos (may be NULL) as in sg_solve_batch.  Returns SG_OK or
 * the first failing system's status; SG_E_ARG for unsupported options before any work. */
int sg_solve_batch_graph(sg_handle* hs, const double* const* F, double* const* U, int nsys, const sg_solve_opts* opts,
                         sg_solve_info* infos);
/* sg_solve_batch_graph in three calls, for a batch solved repeatedly: sg_batch_create does the checks,
 * the workspaces and the graph construction (same arguments as sg_solve_batch_graph; *out receives the
 * batch); sg_batch_solve solves it (U[s] overwritten, infos as above); sg_batch_destroy releases the
 * graphs.  Between create and destroy the handles' workspaces must not change: a solve with a larger
 * restart or another precision on one of them makes sg_batch_solve return SG_E_STATE. */
typedef struct sg_batch_ctx* sg_batch;
int sg_batch_create(sg_handle* hs, const double* const* F, double* const* U, int nsys, const sg_solve_opts* opts,
                    sg_batch* out);
int sg_batch_solve(sg_batch b, sg_solve_info* infos);
void sg_batch_destroy(sg_batch b);

/* Choose the operator kernel's tile (the number of grid rows a warp walks) for this
 * problem by timing the candidates 4, 8, 16, 32 and 64 on the device (a tuning step of
 * this implementation; the paper has no counterpart).  which: bit 0 FP64 arithmetic,
 * bit 1 FP32, bit 2 double-float; 0 = all.  Allocates two temporary vectors of P*N_x
 * doubles and runs about sixty operator applications on the handle's stream; the
 * choice is kept in the handle and cached for the process by (n, M, p, couplings,
 * mean), so later handles of the same shape are tuned without timing.  Without this
 * call the tile is 16 rows. */
int sg_autotune(sg_handle h, int which);

/* Objective J = E[Q] + Var[Q]/2, Q = int u dx: J = m^T U_0 + 1/2 sum_{i>=1}(m^T U_i)^2
 * with m_s = h^2, and its gradient G = dJ/dU (device U, G; J host). */
int sg_objective(sg_handle h, const double* U, double* J, double* G);
/* Adjoint gradients: g_abar[e] = -sum_i Lam_i|e^T K_ref U_i|e (dJ/dabar per
 * cell, device, (n-1)^2 values) and *g_sigma = -(1/sigma) Lam^T (A - I (x) K_0) U
 * (host), given the forward solution U and the adjoint Lam (device FP64). */
int sg_adjoint_gradients(sg_handle h, const double* U, const double* Lam, double sigma,
                         double* g_abar, double* g_sigma);

/* Tracing (no counterpart in the paper): per-phase device time measured with
 * CUDA events recorded on the handle's stream around the kernels of each phase
 * of sg_solve.  Phases: 0 = outer operator A z (FP64), 1 = preconditioner
 * (sweep + V-cycles), 2 = Gram-Schmidt kernels, 3 = other vector kernels.
 * sg_timing_enable(h, 1) starts a fresh accumulation (0 stops recording).
 * sg_timing_read synchronises the stream and writes the accumulated ms[4] and
 * kernel-launch counts launches[4] since the last enable/read (either pointer
 * may be NULL), then resets them.  Kernel launches are counted whether or not
 * timing is enabled. */
int sg_timing_enable(sg_handle h, int enable);
int sg_timing_read(sg_handle h, double* ms, long long* launches);

#ifdef __cplusplus
}
#endif
#endif
