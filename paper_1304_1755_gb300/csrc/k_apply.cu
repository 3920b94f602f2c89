// K1: matrix-free SG operator  Y_i = sum_k sum_j G_k(i,j) K_k X_j  (Eq. tensor-product),
// and its restriction to the lower / upper degree couplings (the stage update of the
// block-triangular sweep, Sec. 4.2).
//
// Q1 element matrix of the Laplacian on a square cell, corners SW(a) SE(b) NE(c) NW(d):
//   K_ref = (1/6)[4 -1 -2 -1; -1 4 -1 -2; -2 -1 4 -1; -1 -2 -1 4]
//         = (1/2) f1 f1^T + (1/2) f2 f2^T + (1/6) f3 f3^T,
//   f1 = (1,0,-1,0), f2 = (0,1,0,-1), f3 = (1,-1,1,-1).
// So K_ref x is fixed by three cell features d1 = xa - xc, d2 = xb - xd,
// hg = xa - xb + xc - xd, and K_k X_j = sum_e c_k(e) K_ref^(e) X_j is linear in them.
// Per output row i and cell e the kernel mixes the features of every coupled
// column j with weight c_k(e) G_k(i,j), then scatters the mixed features to the
// four corners:  a += A + C, b += B - C, c += -A + C, d += -B - C  with
// A = D1/2, B = D2/2, C = H/6.
//
// Launch: CTA = 32 x 8 output nodes (33 x 9 cells) and ROWS_PER_CTA output rows;
// the 1-D grid enumerates (tile, row group) with row groups fastest, so a tile's
// input columns are reused from L2 by neighbouring CTAs.
#include "sg_internal.h"

namespace {
constexpr int TX = 32, TY = 8, CX = TX + 1, CY = TY + 1, NCELL = CX * CY, NT = TX * TY;
constexpr int ROWS_PER_CTA = 4;

template <typename TX_, typename TA>
__device__ __forceinline__ TA ldx(const TX_* X, int vx, int vy, int n, int m) {
  return (vx >= 1 && vx <= n - 2 && vy >= 1 && vy <= n - 2) ? ld_as<TA>(X + (size_t)(vx - 1) + (size_t)(vy - 1) * m)
                                                            : TA(0);
}

template <typename TXS, typename TYS, typename TA, bool EPI>
__global__ void __launch_bounds__(NT) k_apply(const TXS* __restrict__ X, TYS* __restrict__ Y,
                                              const double* __restrict__ R, const TA* __restrict__ coef,
                                              const int* __restrict__ row_ptr, const int* __restrict__ tj,
                                              const int* __restrict__ tk, const TA* __restrict__ tg, int row0,
                                              int nrows, int ybase, int rbase, int n, int m, size_t Nx, size_t Nc,
                                              int tiles_x, int ngroups) {
  __shared__ TA sA[NCELL], sB[NCELL], sC[NCELL];
  const int tid = threadIdx.x;
  const int tile = blockIdx.x / ngroups, group = blockIdx.x % ngroups;   // row groups vary fastest
  const int X0 = (tile % tiles_x) * TX, Y0 = (tile / tiles_x) * TY;     // interior node origin
  const int rbeg = row0 + group * ROWS_PER_CTA;
  const int rend = min(rbeg + ROWS_PER_CTA, row0 + nrows);
  for (int i = rbeg; i < rend; ++i) {
    const int t0 = row_ptr[i], t1 = row_ptr[i + 1];
    for (int c = tid; c < NCELL; c += NT) {
      const int cx = X0 + (c % CX), cy = Y0 + (c / CX);    // cell coordinates
      TA a0 = 0, a1 = 0, a2 = 0;
      if (cx <= n - 2 && cy <= n - 2) {
        const size_t e = (size_t)cx + (size_t)cy * (n - 1);
        for (int t = t0; t < t1; ++t) {
          const TXS* Xj = X + (size_t)tj[t] * Nx;
          const TA w = coef[(size_t)tk[t] * Nc + e] * tg[t];
          const TA xa = ldx<TXS, TA>(Xj, cx, cy, n, m);
          const TA xb = ldx<TXS, TA>(Xj, cx + 1, cy, n, m);
          const TA xc = ldx<TXS, TA>(Xj, cx + 1, cy + 1, n, m);
          const TA xd = ldx<TXS, TA>(Xj, cx, cy + 1, n, m);
          a0 += w * (xa - xc);
          a1 += w * (xb - xd);
          a2 += w * ((xa + xc) - (xb + xd));
        }
      }
      sA[c] = a0 * TA(0.5);
      sB[c] = a1 * TA(0.5);
      sC[c] = a2 * (TA(1) / TA(6));
    }
    __syncthreads();
    const int tx = tid % TX, ty = tid / TX;
    const int ix = X0 + tx, iy = Y0 + ty;
    if (ix < m && iy < m) {
      const int cNE = tx + ty * CX;              // node is the NE corner of this cell
      const int cNW = (tx + 1) + ty * CX;        // node is the NW corner
      const int cSE = tx + (ty + 1) * CX;        // node is the SE corner
      const int cSW = (tx + 1) + (ty + 1) * CX;  // node is the SW corner
      TA y = (sA[cSW] + sC[cSW]) + (sB[cSE] - sC[cSE]) + (sC[cNE] - sA[cNE]) - (sB[cNW] + sC[cNW]);
      const size_t s = (size_t)ix + (size_t)iy * m;
      if (EPI) y = (TA)R[(size_t)(i - rbase) * Nx + s] - y;
      st_as<TYS, TA>(Y + (size_t)(i - ybase) * Nx + s, y);
    }
    __syncthreads();
  }
}

template <typename TXS, typename TYS, typename TA>
int launch_t(sg_ctx* h, const TermTable& T, const TXS* X, TYS* Y, const double* R, int row0, int nrows, int ybase,
             int rbase) {
  if (nrows <= 0) return SG_OK;
  const int tiles_x = (h->m + TX - 1) / TX, tiles_y = (h->m + TY - 1) / TY;
  const int ngroups = (nrows + ROWS_PER_CTA - 1) / ROWS_PER_CTA;
  const unsigned grid = (unsigned)ngroups * (unsigned)(tiles_x * tiles_y);
  const TA* coef = nullptr;
  const TA* tg = nullptr;
  if constexpr (sizeof(TA) == 8) { coef = (const TA*)h->coef64; tg = (const TA*)T.g; }
  else { coef = (const TA*)h->coef32; tg = (const TA*)T.gf; }
  if (R)
    k_apply<TXS, TYS, TA, true><<<grid, NT, 0, h->stream>>>(X, Y, R, coef, T.row_ptr, T.j, T.k, tg, row0, nrows, ybase,
                                                             rbase, h->n, h->m, h->Nx, h->Nc, tiles_x, ngroups);
  else
    k_apply<TXS, TYS, TA, false><<<grid, NT, 0, h->stream>>>(X, Y, R, coef, T.row_ptr, T.j, T.k, tg, row0, nrows,
                                                              ybase, rbase, h->n, h->m, h->Nx, h->Nc, tiles_x, ngroups);
  SG_CUDA(h, cudaGetLastError());
  count_launch(h);
  return SG_OK;
}

template <typename TA>
int dispatch_y(sg_ctx* h, const TermTable& T, int xprec, const void* X, int yprec, void* Y, const double* R, int row0,
               int nrows, int ybase, int rbase) {
#define SG_Y(TXS)                                                                                             \
  switch (yprec) {                                                                                            \
    case SG_F64: return launch_t<TXS, double, TA>(h, T, (const TXS*)X, (double*)Y, R, row0, nrows, ybase, rbase); \
    case SG_F32: return launch_t<TXS, float, TA>(h, T, (const TXS*)X, (float*)Y, R, row0, nrows, ybase, rbase);   \
    case SG_BF16: return launch_t<TXS, bf16, TA>(h, T, (const TXS*)X, (bf16*)Y, R, row0, nrows, ybase, rbase);    \
  }
  switch (xprec) {
    case SG_F64: SG_Y(double) break;
    case SG_F32: SG_Y(float) break;
    case SG_BF16: SG_Y(bf16) break;
  }
#undef SG_Y
  return sg_fail(h, SG_E_ARG, "apply: bad precision");
}
}  // namespace

int launch_apply(sg_ctx* h, int which, int xprec, const void* X, int yprec, void* Y, const double* R, int row0,
                 int nrows, int ybase, int rbase, int arith64) {
  const TermTable& T = which == 0 ? h->t_all : (which == 1 ? h->t_lower : (which == 2 ? h->t_upper : h->t_off));
  if (arith64) return dispatch_y<double>(h, T, xprec, X, yprec, Y, R, row0, nrows, ybase, rbase);
  return dispatch_y<float>(h, T, xprec, X, yprec, Y, R, row0, nrows, ybase, rbase);
}
