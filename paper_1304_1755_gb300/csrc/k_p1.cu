// The paper's own discretisation on the GPU (Sec. 6): linear elements on the uniform triangulation
// with SW-NE diagonals, the coefficient constant per triangle, and one point Gauss-Seidel V-cycle per
// diagonal block.
//
// Operator.  On these right triangles the element matrix couples only the two ends of each leg (the
// diagonal's ends have orthogonal gradients), so K_k is a graph Laplacian on the grid's edges:
//   (K_k z)_v = sum over the four edges e = (v, u) of w_k(e) (z_v - z_u),   z_u = 0 on the boundary,
// with w_k(e) = (c_k(T) + c_k(T')) / 2 over the two triangles sharing the edge (lower-right triangle of
// cell (x, y) and upper-left triangle of cell (x, y-1) for the horizontal edge (x, y)-(x+1, y); upper-left
// of (x, y) and lower-right of (x-1, y) for the vertical edge (x, y)-(x, y+1)).  One thread per node and
// output row; FP64.
//
// V-cycle.  With the mean coefficient 1 every level is the 5-point Laplacian (4, -1) (Galerkin products
// with linear interpolation on nested triangulations reproduce it).  One CTA runs the whole cycle of one
// block from a zero guess: nu1 forward Gauss-Seidel sweeps, the residual, its restriction by P^T
// (weights 1 at the coarse node, 1/2 at the four axis neighbours and at the NE and SW diagonal
// neighbours), the coarser levels, the coarsest (one node) solved exactly, then the prolongation and nu2
// backward sweeps.  Red-black order: a half-sweep updates all nodes of one colour at once.  Lexicographic
// order: a node is updated from the new values of its west and south neighbours and the old values of
// its east and north ones, so the nodes of one anti-diagonal are independent and the sweep runs as
// 2m - 1 wavefronts separated by CTA barriers.  Level data live in a per-block global workspace
// (L2-resident at the paper's sizes).
#include <algorithm>
#include <vector>

#include "sg_internal.h"

namespace {
constexpr int P1_THREADS = 1024;

struct P1Args {
  const double* X;
  double* Y;
  const double* R;
  const double* ew;          // (M+1) x 2 x n^2: horizontal weights then vertical, vertex-indexed
  const int* row_ptr;
  const int* tj;
  const int* tk;
  const double* tg;
  int row0, ybase, rbase, n, m;
  size_t Nx;
};

__global__ void k_apply_p1(P1Args a) {
  const int i = a.row0 + blockIdx.y;
  const size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (s >= a.Nx) return;
  const int m = a.m, n = a.n;
  const int ix = (int)(s % m), iy = (int)(s / m);
  const int vx = ix + 1, vy = iy + 1;                    // vertex of the node
  const size_t nn = (size_t)n * n;
  double acc = 0.0;
  for (int t = a.row_ptr[i]; t < a.row_ptr[i + 1]; ++t) {
    const double* z = a.X + (size_t)a.tj[t] * a.Nx;
    const double* wh = a.ew + (size_t)a.tk[t] * 2 * nn;
    const double* wv = wh + nn;
    const double zc = z[s];
    const double zw = ix > 0 ? z[s - 1] : 0.0, ze = ix < m - 1 ? z[s + 1] : 0.0;
    const double zs = iy > 0 ? z[s - m] : 0.0, zn = iy < m - 1 ? z[s + m] : 0.0;
    const double k = wh[(size_t)vy * n + vx - 1] * (zc - zw) + wh[(size_t)vy * n + vx] * (zc - ze) +
                     wv[(size_t)(vy - 1) * n + vx] * (zc - zs) + wv[(size_t)vy * n + vx] * (zc - zn);
    acc += a.tg[t] * k;
  }
  const size_t yo = (size_t)(i - a.ybase) * a.Nx + s;
  a.Y[yo] = a.R ? a.R[(size_t)(i - a.rbase) * a.Nx + s] - acc : acc;
}

struct P1Levels {
  int nl;
  int m[SG_MAX_LEVELS];
  size_t xo[SG_MAX_LEVELS], bo[SG_MAX_LEVELS], ro[SG_MAX_LEVELS];   // offsets in the block's workspace
};

__device__ __forceinline__ void gs_node(double* x, const double* b, int m, int i, int j) {
  const size_t t = (size_t)j * m + i;
  double sn = b[t];
  if (i > 0) sn += x[t - 1];
  if (i < m - 1) sn += x[t + 1];
  if (j > 0) sn += x[t - m];
  if (j < m - 1) sn += x[t + m];
  x[t] = 0.25 * sn;
}

// one Gauss-Seidel sweep of the 5-point Laplacian (4, -1) on an m x m level, lexicographic or red-black
__device__ void gs_sweep(double* x, const double* b, int m, bool forward, bool redblack) {
  if (redblack) {
    const int hm = (m + 1) / 2;                           // nodes of one colour in a row, at most
    for (int h = 0; h < 2; ++h) {
      const int c = forward ? h : 1 - h;
      for (int q = threadIdx.x; q < hm * m; q += blockDim.x) {
        const int j = q / hm, i = 2 * (q % hm) + ((j + c) & 1);
        if (i < m) gs_node(x, b, m, i, j);
      }
      __syncthreads();
    }
    return;
  }
  for (int w = 0; w <= 2 * (m - 1); ++w) {
    const int d = forward ? w : 2 * (m - 1) - w;
    const int i0 = max(0, d - (m - 1)), i1 = min(d, m - 1);
    for (int q = threadIdx.x; q <= i1 - i0; q += blockDim.x) gs_node(x, b, m, i0 + q, d - i0 - q);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(P1_THREADS) k_p1_vcycle(const double* __restrict__ B, size_t ldb,
                                                          double* X, size_t ldx, double* W, size_t ldw,
                                                          P1Levels L, int nu1, int nu2, bool rb) {
  const int blk = blockIdx.x;
  double* w = W + (size_t)blk * ldw;
  auto xl = [&](int l) -> double* { return l == 0 ? X + (size_t)blk * ldx : w + L.xo[l]; };
  auto bl = [&](int l) -> const double* { return l == 0 ? B + (size_t)blk * ldb : w + L.bo[l]; };
  for (int l = 0; l + 1 < L.nl; ++l) {
    const int m = L.m[l], mc = L.m[l + 1];
    double* x = xl(l);
    const double* b = bl(l);
    double* r = w + L.ro[l];
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) x[t] = 0.0;
    __syncthreads();
    for (int s = 0; s < nu1; ++s) gs_sweep(x, b, m, true, rb);
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
      const int i = t % m, j = t / m;
      double ax = 4.0 * x[t];
      if (i > 0) ax -= x[t - 1];
      if (i < m - 1) ax -= x[t + 1];
      if (j > 0) ax -= x[t - m];
      if (j < m - 1) ax -= x[t + m];
      r[t] = b[t] - ax;
    }
    __syncthreads();
    // coarse node (I, J) sits on fine interior node (2I + 1, 2J + 1); every neighbour below is inside
    double* bc = w + L.bo[l + 1];
    for (int t = threadIdx.x; t < mc * mc; t += blockDim.x) {
      const int I = t % mc, J = t / mc;
      const size_t f = (size_t)(2 * J + 1) * m + (2 * I + 1);
      bc[t] = r[f] + 0.5 * (r[f - 1] + r[f + 1] + r[f - m] + r[f + m] + r[f + m + 1] + r[f - m - 1]);
    }
    __syncthreads();
  }
  {
    const int l = L.nl - 1;                               // one node: A = 4
    if (threadIdx.x == 0) xl(l)[0] = 0.25 * bl(l)[0];
    __syncthreads();
  }
  for (int l = L.nl - 2; l >= 0; --l) {
    const int m = L.m[l], mc = L.m[l + 1];
    double* x = xl(l);
    const double* xc = xl(l + 1);
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
      const int i = t % m, j = t / m;
      // fine interior (i, j) = vertex (i + 1, j + 1); coarse interior (I, J) = vertex (2I + 2, 2J + 2)
      auto c = [&](int I, int J) { return (I >= 0 && I < mc && J >= 0 && J < mc) ? xc[(size_t)J * mc + I] : 0.0; };
      double e;
      if ((i & 1) && (j & 1)) e = c((i - 1) / 2, (j - 1) / 2);                  // on a coarse node
      else if (j & 1) e = 0.5 * (c(i / 2 - 1, (j - 1) / 2) + c(i / 2, (j - 1) / 2));   // horizontal edge
      else if (i & 1) e = 0.5 * (c((i - 1) / 2, j / 2 - 1) + c((i - 1) / 2, j / 2));   // vertical edge
      else e = 0.5 * (c(i / 2 - 1, j / 2 - 1) + c(i / 2, j / 2));               // SW-NE diagonal
      x[t] += e;
    }
    __syncthreads();
    for (int s = 0; s < nu2; ++s) gs_sweep(x, bl(l), m, false, rb);
  }
}
}  // namespace

int setup_p1(sg_ctx* h) {
  const int n = h->n, nc1 = n - 1, M = h->M;
  const size_t nn = (size_t)n * n, Nt = 2 * (size_t)nc1 * nc1;
  for (size_t e = 0; e < Nt; ++e)
    if (h->coef_h[e] != 1.0) return sg_fail(h, SG_E_ARG, "P1 elements need the mean coefficient 1 on every triangle");
  // c(T) of a cell's lower-right (0) or upper-left (1) triangle, 0 outside the grid of cells
  auto ct = [&](int k, int cx, int cy, int tri) {
    if (cx < 0 || cx >= nc1 || cy < 0 || cy >= nc1) return 0.0;
    return h->coef_h[(size_t)k * Nt + 2 * ((size_t)cy * nc1 + cx) + tri];
  };
  std::vector<double> ew((size_t)(M + 1) * 2 * nn, 0.0);
  for (int k = 0; k <= M; ++k) {
    double* wh = ew.data() + (size_t)k * 2 * nn;
    double* wv = wh + nn;
    for (int y = 0; y < n; ++y)
      for (int x = 0; x < n; ++x) {
        wh[(size_t)y * n + x] = 0.5 * (ct(k, x, y, 0) + ct(k, x, y - 1, 1));     // edge (x, y)-(x+1, y)
        wv[(size_t)y * n + x] = 0.5 * (ct(k, x, y, 1) + ct(k, x - 1, y, 0));     // edge (x, y)-(x, y+1)
      }
  }
  if (cudaMalloc(&h->ew, sizeof(double) * ew.size()) != cudaSuccess) return sg_fail(h, SG_E_ALLOC, "P1 edge weights");
  SG_CUDA(h, cudaMemcpy(h->ew, ew.data(), sizeof(double) * ew.size(), cudaMemcpyHostToDevice));
  // per-block workspace: level 0 residual; levels >= 1 solution, right-hand side and residual
  size_t ld = 0;
  for (int l = 0; l < h->nlev; ++l) ld += (l == 0 ? 1 : 3) * h->lev[l].N;
  h->p1w_ld = (ld + 31) / 32 * 32;
  if (cudaMalloc(&h->p1w, sizeof(double) * h->p1w_ld * h->P) != cudaSuccess)
    return sg_fail(h, SG_E_ALLOC, "P1 multigrid workspace");
  return SG_OK;
}

int launch_apply_p1(sg_ctx* h, int which, int xprec, const void* X, int yprec, void* Y, int rprec, const void* R,
                    int row0, int nrows, int ybase, int rbase, int arith) {
  if (xprec != SG_F64 || yprec != SG_F64 || arith != SG_F64 || (R && rprec != SG_F64))
    return sg_fail(h, SG_E_ARG, "P1 elements: FP64 operators only");
  if (nrows <= 0) return SG_OK;
  const TermTable& T = which == 0 ? h->t_all : which == 1 ? h->t_lower : which == 2 ? h->t_upper
                                                            : which == 3 ? h->t_off : h->t_diag;
  P1Args a{};
  a.X = (const double*)X, a.Y = (double*)Y, a.R = (const double*)R, a.ew = h->ew;
  a.row_ptr = T.row_ptr, a.tj = T.j, a.tk = T.k, a.tg = T.g;
  a.row0 = row0, a.ybase = ybase, a.rbase = rbase, a.n = h->n, a.m = h->m, a.Nx = h->Nx;
  const dim3 grid((unsigned)((h->Nx + 255) / 256), (unsigned)nrows);
  k_apply_p1<<<grid, 256, 0, h->stream>>>(a);
  SG_CUDA(h, cudaGetLastError());
  count_launch(h);
  return SG_OK;
}

int vcycle_p1(sg_ctx* h, int nb, const double* B, size_t ldb, double* X, size_t ldx) {
  if (nb <= 0) return SG_OK;
  P1Levels L{};
  L.nl = h->nlev;
  size_t off = 0;
  for (int l = 0; l < h->nlev; ++l) {
    L.m[l] = h->lev[l].m;
    L.ro[l] = off;
    off += h->lev[l].N;
    if (l > 0) {
      L.xo[l] = off, off += h->lev[l].N;
      L.bo[l] = off, off += h->lev[l].N;
    }
  }
  k_p1_vcycle<<<nb, P1_THREADS, 0, h->stream>>>(B, ldb, X, ldx, h->p1w, h->p1w_ld, L, h->nu1, h->nu2,
                                                      h->gs_order == SG_GS_RB);
  SG_CUDA(h, cudaGetLastError());
  count_launch(h);
  return SG_OK;
}
