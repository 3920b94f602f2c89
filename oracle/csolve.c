/*
 * Plain FP64 C implementation of the oracle's block-triangular preconditioned flexible GMRES
 * (TEST INFRASTRUCTURE ONLY: used by the tests and by the CPU-baseline leg of the benchmark,
 * never by the CUDA library).  It runs the same steps as the Python oracle, in the same order,
 * on all host cores through OpenMP parallel loops; the matrices come from the Python oracle
 * (oracle.sg.build and oracle.mg.Hierarchy) as CSR arrays, so this file holds no assembly.
 *
 *   operator   Y_i = sum over the terms (j, k, g) of PC row i of g K_k X_j
 *              (Eq. tensor-product: A = sum_k G_k (x) K_k, G_0 = I)
 *   B_T^{-1}   for i = 0 .. P-1: T = R_i - sum over the lower terms (j < i) of g K_k Z_j,
 *              Z_i = V-cycle(T)  (Sec. 4.2: block forward substitution, diagonal blocks K_0
 *              approximated by one multigrid V-cycle); B_T^{-T}: i = P-1 .. 0 over the
 *              transposed upper terms (j > i) of A^T (the adjoint solve)
 *   V-cycle    from zero: nu1 damped-Jacobi steps x += omega D^{-1}(b - A x), restriction of
 *              the residual by R = P^T, recursion, prolongation x += P x_c, nu2 Jacobi steps;
 *              the coarsest level by its dense inverse (Sec. 4.1, 6)
 *   FGMRES     right-preconditioned restarted flexible GMRES (Saad-Schultz, cited in Sec. 4.2),
 *              modified Gram-Schmidt, Givens rotations, x0 = 0, the true residual recomputed at
 *              every restart, stop when ||F - A U|| <= tol ||F||
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC csolve.c -o libsgo.so (oracle/cbuild.py).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int nrows;
  const int* ptr;
  const int* idx;
  const double* val;
} sgo_csr;

typedef struct {
  int P, Nx, M;
  const sgo_csr* K;            /* M + 1 stiffness matrices K_k (Nx x Nx) */
  const int* t_ptr;            /* all terms of A, CSR over the P rows: column j, mode k, value g */
  const int* t_j;
  const int* t_k;
  const double* t_g;
  const int* l_ptr;            /* the terms with j < i (the strictly lower blocks of A) */
  const int* l_j;
  const int* l_k;
  const double* l_g;
  const int* u_ptr;            /* the terms of A^T with j > i (its strictly upper blocks): row i holds */
  const int* u_j;              /* (j, k, G_k(j, i)) so that (A^T)_ij = sum G_k(j, i) K_k^T and */
  const int* u_k;              /* K_k^T = K_k (symmetric stiffness matrices) */
  const double* u_g;
  int nlev;                    /* multigrid levels, 0 = fine */
  const sgo_csr* A;            /* nlev level operators (A_0 = K_0) */
  const double* const* Dinv;   /* nlev inverse diagonals */
  const sgo_csr* Pr;           /* nlev - 1 prolongations, level l+1 -> l (N_l x N_{l+1}) */
  const sgo_csr* Rs;           /* nlev - 1 restrictions P_l^T (N_{l+1} x N_l) */
  const double* coarse_inv;    /* dense inverse of the coarsest operator, row-major */
  int nu1, nu2;
  double omega;
} sgo_problem;

int sgo_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* y = A x */
static void spmv(const sgo_csr* A, const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int r = 0; r < A->nrows; ++r) {
    double s = 0.0;
    for (int q = A->ptr[r]; q < A->ptr[r + 1]; ++q) s += A->val[q] * x[A->idx[q]];
    y[r] = s;
  }
}

/* y += A x */
static void spmv_add(const sgo_csr* A, const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int r = 0; r < A->nrows; ++r) {
    double s = 0.0;
    for (int q = A->ptr[r]; q < A->ptr[r + 1]; ++q) s += A->val[q] * x[A->idx[q]];
    y[r] += s;
  }
}

/* One V(nu1, nu2) cycle from a zero guess on level l: x = V_l(b).  work holds 3 N_l doubles per
 * level at offsets woff[l]. */
static void vcycle(const sgo_problem* pb, int l, const double* b, double* x, double* work, const size_t* woff) {
  const sgo_csr* A = &pb->A[l];
  const int N = A->nrows;
  if (l == pb->nlev - 1) {
#pragma omp parallel for schedule(static)
    for (int r = 0; r < N; ++r) {
      double s = 0.0;
      for (int c = 0; c < N; ++c) s += pb->coarse_inv[(size_t)r * N + c] * b[c];
      x[r] = s;
    }
    return;
  }
  double* ax = work + woff[l];
  double* bc = ax + N;
  double* xc = bc + pb->A[l + 1].nrows;
  const double* dinv = pb->Dinv[l];
  const double w = pb->omega;
  memset(x, 0, sizeof(double) * (size_t)N);
  for (int s = 0; s < pb->nu1; ++s) {
    spmv(A, x, ax);
#pragma omp parallel for schedule(static)
    for (int r = 0; r < N; ++r) x[r] += w * dinv[r] * (b[r] - ax[r]);
  }
  spmv(A, x, ax);
#pragma omp parallel for schedule(static)
  for (int r = 0; r < N; ++r) ax[r] = b[r] - ax[r];          /* residual */
  spmv(&pb->Rs[l], ax, bc);                                  /* b_c = P^T r */
  vcycle(pb, l + 1, bc, xc, work, woff);
  spmv_add(&pb->Pr[l], xc, x);                               /* x += P x_c */
  for (int s = 0; s < pb->nu2; ++s) {
    spmv(A, x, ax);
#pragma omp parallel for schedule(static)
    for (int r = 0; r < N; ++r) x[r] += w * dinv[r] * (b[r] - ax[r]);
  }
}

static size_t* vcycle_offsets(const sgo_problem* pb, size_t* total) {
  size_t* off = (size_t*)malloc(sizeof(size_t) * (size_t)pb->nlev);
  size_t t = 0;
  for (int l = 0; l < pb->nlev; ++l) {
    off[l] = t;
    if (l + 1 < pb->nlev) t += 2 * (size_t)pb->A[l].nrows + (size_t)pb->A[l + 1].nrows;
  }
  *total = t;
  return off;
}

/* Y = A X: each PC row's terms, one node at a time */
void sgo_apply(const sgo_problem* pb, const double* X, double* Y) {
  const int P = pb->P, Nx = pb->Nx;
  const long long NN = (long long)P * Nx;
#pragma omp parallel for schedule(static)
  for (long long q = 0; q < NN; ++q) {
    const int i = (int)(q / Nx), s = (int)(q % Nx);
    double acc = 0.0;
    for (int t = pb->t_ptr[i]; t < pb->t_ptr[i + 1]; ++t) {
      const sgo_csr* K = &pb->K[pb->t_k[t]];
      const double* xj = X + (size_t)pb->t_j[t] * Nx;
      double ks = 0.0;
      for (int c = K->ptr[s]; c < K->ptr[s + 1]; ++c) ks += K->val[c] * xj[K->idx[c]];
      acc += pb->t_g[t] * ks;
    }
    Y[q] = acc;
  }
}

/* one V-cycle on each of nb stacked blocks (B_D^{-1} for nb = P) */
void sgo_vcycles(const sgo_problem* pb, int nb, const double* B, double* X) {
  size_t tot;
  size_t* woff = vcycle_offsets(pb, &tot);
  double* work = (double*)malloc(sizeof(double) * (tot + 1));
  for (int b = 0; b < nb; ++b) vcycle(pb, 0, B + (size_t)b * pb->Nx, X + (size_t)b * pb->Nx, work, woff);
  free(work);
  free(woff);
}

/* Z = B_T^{-1} R by block forward substitution over the PC rows, or Z = B_T^{-T} R by backward
 * substitution (transpose != 0) */
void sgo_precond_bt(const sgo_problem* pb, const double* R, double* Z, int transpose) {
  const int P = pb->P, Nx = pb->Nx;
  const int* tp = transpose ? pb->u_ptr : pb->l_ptr;
  const int* tj = transpose ? pb->u_j : pb->l_j;
  const int* tk = transpose ? pb->u_k : pb->l_k;
  const double* tg = transpose ? pb->u_g : pb->l_g;
  size_t tot;
  size_t* woff = vcycle_offsets(pb, &tot);
  double* work = (double*)malloc(sizeof(double) * (tot + 1));
  double* T = (double*)malloc(sizeof(double) * (size_t)Nx);
  for (int step = 0; step < P; ++step) {
    const int i = transpose ? P - 1 - step : step;
#pragma omp parallel for schedule(static)
    for (int s = 0; s < Nx; ++s) {
      double acc = R[(size_t)i * Nx + s];
      for (int t = tp[i]; t < tp[i + 1]; ++t) {
        const sgo_csr* K = &pb->K[tk[t]];
        const double* zj = Z + (size_t)tj[t] * Nx;
        double ks = 0.0;
        for (int c = K->ptr[s]; c < K->ptr[s + 1]; ++c) ks += K->val[c] * zj[K->idx[c]];
        acc -= tg[t] * ks;
      }
      T[s] = acc;
    }
    vcycle(pb, 0, T, Z + (size_t)i * Nx, work, woff);
  }
  free(T);
  free(work);
  free(woff);
}

static double dot(const double* x, const double* y, size_t N) {
  double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (long long q = 0; q < (long long)N; ++q) s += x[q] * y[q];
  return s;
}

/* Flexible GMRES(restart) with B_T^{-1}, x0 = 0; with transpose != 0 the adjoint system
 * A^T U = F with B_T^{-T} (A = A^T here: G_k and K_k are symmetric, so only the sweep changes).
 * Returns 0 on convergence, 1 at maxit, -1 on a non-finite value or allocation failure.
 * *iters = preconditioner applications. */
int sgo_bt_fgmres(const sgo_problem* pb, const double* F, double* U, int restart, int maxit, double tol,
                  int transpose, int* iters, double* relres) {
  const size_t N = (size_t)pb->P * pb->Nx;
  const int m = restart;
  double* V = (double*)malloc(sizeof(double) * N * (size_t)(m + 1));
  double* Zs = (double*)malloc(sizeof(double) * N * (size_t)m);
  double* w = (double*)malloc(sizeof(double) * N);
  double* H = (double*)calloc((size_t)(m + 1) * m, sizeof(double));
  double* cs = (double*)calloc((size_t)m, sizeof(double));
  double* sn = (double*)calloc((size_t)m, sizeof(double));
  double* g = (double*)calloc((size_t)m + 1, sizeof(double));
  double* y = (double*)calloc((size_t)m, sizeof(double));
  int rc = 0, its = 0;
  if (!V || !Zs || !w || !H || !cs || !sn || !g || !y) { rc = -1; goto done; }
  memset(U, 0, sizeof(double) * N);
  const double bnorm = sqrt(dot(F, F, N));
  *relres = 0.0;
  if (bnorm == 0.0) goto done;
  for (;;) {
    /* true residual r = F - A U into V_0 */
    sgo_apply(pb, U, w);
#pragma omp parallel for schedule(static)
    for (long long q = 0; q < (long long)N; ++q) V[q] = F[q] - w[q];
    const double beta = sqrt(dot(V, V, N));
    if (!isfinite(beta)) { rc = -1; break; }
    *relres = beta / bnorm;
    if (beta <= tol * bnorm) break;
    if (its >= maxit) { rc = 1; break; }
#pragma omp parallel for schedule(static)
    for (long long q = 0; q < (long long)N; ++q) V[q] /= beta;
    memset(g, 0, sizeof(double) * ((size_t)m + 1));
    g[0] = beta;
    int k = 0;
    for (int j = 0; j < m; ++j) {
      double* zj = Zs + (size_t)j * N;
      sgo_precond_bt(pb, V + (size_t)j * N, zj, transpose);
      sgo_apply(pb, zj, w);
      for (int i = 0; i <= j; ++i) {                       /* modified Gram-Schmidt */
        const double* vi = V + (size_t)i * N;
        const double hij = dot(vi, w, N);
        H[(size_t)i * m + j] = hij;
#pragma omp parallel for schedule(static)
        for (long long q = 0; q < (long long)N; ++q) w[q] -= hij * vi[q];
      }
      const double hn = sqrt(dot(w, w, N));
      H[(size_t)(j + 1) * m + j] = hn;
      for (int i = 0; i < j; ++i) {                        /* earlier rotations on column j */
        const double a = H[(size_t)i * m + j], b = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * b;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * b;
      }
      const double d = hypot(H[(size_t)j * m + j], H[(size_t)(j + 1) * m + j]);
      if (!isfinite(d) || d == 0.0) { rc = -1; goto done; }
      cs[j] = H[(size_t)j * m + j] / d;
      sn[j] = H[(size_t)(j + 1) * m + j] / d;
      H[(size_t)j * m + j] = d;
      H[(size_t)(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++its;
      k = j + 1;
      if (fabs(g[j + 1]) <= tol * bnorm || its >= maxit || hn == 0.0) break;
      double* vn = V + (size_t)(j + 1) * N;
#pragma omp parallel for schedule(static)
      for (long long q = 0; q < (long long)N; ++q) vn[q] = w[q] / hn;
    }
    for (int i = k - 1; i >= 0; --i) {                     /* back substitution */
      double s = g[i];
      for (int l = i + 1; l < k; ++l) s -= H[(size_t)i * m + l] * y[l];
      y[i] = s / H[(size_t)i * m + i];
    }
    for (int i = 0; i < k; ++i) {                          /* U += Z y */
      const double* zi = Zs + (size_t)i * N;
      const double yi = y[i];
#pragma omp parallel for schedule(static)
      for (long long q = 0; q < (long long)N; ++q) U[q] += yi * zi[q];
    }
  }
done:
  *iters = its;
  free(V), free(Zs), free(w), free(H), free(cs), free(sn), free(g), free(y);
  return rc;
}
