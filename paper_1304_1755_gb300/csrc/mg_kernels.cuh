// Grid-wide multigrid level kernels (fine levels with n > 33), included by k_mg.cu.
//
// Both kernels work on a shared-memory window of the fine grid and iterate it with a
// 32 x 8 thread layout (x fastest, no integer division).  Out-of-domain window
// points hold 0 (homogeneous Dirichlet boundary).
#pragma once

namespace {
constexpr int MAXNU = 4;
constexpr int CT = 14;                                   // coarse tile of mg_down: fine window 2 CT + 1 + 2 nu1
constexpr int DW = 2 * CT + 1 + 2 * MAXNU;
constexpr int UX = 30, UY = 14;                          // fine tile of mg_up: window (UX + 2H) x (UY + 2H)
constexpr int UH = 2 * MAXNU - 1;
constexpr int UWX = UX + 2 * UH, UWY = UY + 2 * UH;
constexpr int UCX = (UX + 2 * MAXNU) / 2 + 3, UCY = (UY + 2 * MAXNU) / 2 + 3;

#define SG_WLOOP(WX_, WY_)                          \
  for (int lj = ty; lj < (WY_); lj += 8)            \
    for (int li = tx; li < (WX_); li += 32)

// A x at window point (li, lj) of a row-major window of width w (9-point stencil).
template <typename TA, bool VAR>
__device__ __forceinline__ TA apply_pt(const TA* x, int w, int li, int lj, const TA* st) {
  const TA* r0 = x + (lj - 1) * w + li;
  const TA* r1 = r0 + w;
  const TA* r2 = r1 + w;
  if (VAR) {
    return st[0] * r0[-1] + st[1] * r0[0] + st[2] * r0[1] + st[3] * r1[-1] + st[4] * r1[0] + st[5] * r1[1] +
           st[6] * r2[-1] + st[7] * r2[0] + st[8] * r2[1];
  }
  // constant Q1 stencil: 8/3 at the centre, -1/3 at the 8 neighbours
  const TA s9 = (r0[-1] + r0[0] + r0[1]) + (r1[-1] + r1[0] + r1[1]) + (r2[-1] + r2[0] + r2[1]);
  return TA(3) * r1[0] - s9 * (TA(1) / TA(3));
}

template <typename TA, bool VAR>
__device__ __forceinline__ TA dinv_at(const TA* st) {
  if (VAR) return TA(1) / st[4];
  return TA(3) / TA(8);
}

// level l -> l+1: x = S^{nu1}(b) from zero (damped Jacobi), r = b - A x, b_c = P^T r.
template <typename TB, typename TS, typename TA, bool VAR>
__global__ void __launch_bounds__(256) mg_down(const TB* __restrict__ b, TS* __restrict__ bc, int m, int mc,
                                               size_t ldb, size_t ldc, const TA* __restrict__ st, TA omega,
                                               int nu1, int tiles_x) {
  __shared__ TA sb[DW * DW], sx0[DW * DW], sx1[DW * DW];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int tile = blockIdx.x, blk = blockIdx.y;
  const int I0 = (tile % tiles_x) * CT, J0 = (tile / tiles_x) * CT;
  const int W = 2 * CT + 1 + 2 * nu1;
  const int fi0 = 2 * I0 - nu1, fj0 = 2 * J0 - nu1;     // fine interior index of window (0,0)
  const TB* bb = b + (size_t)blk * ldb;
  SG_WLOOP(W, W) {
    const int t = lj * W + li, i = fi0 + li, j = fj0 + lj;
    TA v = 0, xv = 0;
    if (i >= 0 && i < m && j >= 0 && j < m) {
      v = ld_as<TA>(bb + (size_t)i + (size_t)j * m);
      const TA* sp = VAR ? st + 9 * ((size_t)i + (size_t)j * m) : nullptr;
      xv = omega * dinv_at<TA, VAR>(sp) * v;
    }
    sb[t] = v;
    sx0[t] = xv;
  }
  __syncthreads();
  TA* xc = sx0;
  TA* xn = sx1;
  for (int s = 2; s <= nu1; ++s) {
    const int lo = s - 1, hi = W - (s - 1);
    SG_WLOOP(W, W) {
      const int t = lj * W + li, i = fi0 + li, j = fj0 + lj;
      TA v = 0;
      if (li >= lo && li < hi && lj >= lo && lj < hi && i >= 0 && i < m && j >= 0 && j < m) {
        const TA* sp = VAR ? st + 9 * ((size_t)i + (size_t)j * m) : nullptr;
        v = xc[t] + omega * dinv_at<TA, VAR>(sp) * (sb[t] - apply_pt<TA, VAR>(xc, W, li, lj, sp));
      }
      xn[t] = v;
    }
    __syncthreads();
    TA* tmp = xc; xc = xn; xn = tmp;
  }
  {
    // residual on the inner (2 CT + 1)^2 window
    const int lo = nu1, hi = W - nu1;
    SG_WLOOP(W, W) {
      const int t = lj * W + li, i = fi0 + li, j = fj0 + lj;
      TA r = 0;
      if (li >= lo && li < hi && lj >= lo && lj < hi && i >= 0 && i < m && j >= 0 && j < m) {
        const TA* sp = VAR ? st + 9 * ((size_t)i + (size_t)j * m) : nullptr;
        r = sb[t] - apply_pt<TA, VAR>(xc, W, li, lj, sp);
      }
      xn[t] = r;
    }
  }
  __syncthreads();
  // restriction P^T: fine nodes 2I, 2I+1, 2I+2 (interior indices) with weights 1/2, 1, 1/2 per axis
  for (int cj = ty; cj < CT; cj += 8)
    for (int ci = tx; ci < CT; ci += 32) {
      const int I = I0 + ci, J = J0 + cj;
      if (I < mc && J < mc) {
        const int li = 2 * I - fi0, lj = 2 * J - fj0;
        const TA* r0 = xn + lj * W + li;
        const TA* r1 = r0 + W;
        const TA* r2 = r1 + W;
        const TA v = TA(0.25) * (r0[0] + r0[2] + r2[0] + r2[2]) + TA(0.5) * (r0[1] + r1[0] + r1[2] + r2[1]) + r1[1];
        st_as<TS, TA>(bc + (size_t)blk * ldc + (size_t)I + (size_t)J * mc, v);
      }
    }
}

// level l+1 -> l: recompute x_pre = S^{nu1}(b) from zero, x = x_pre + P x_c, nu2 post-smoothing steps.
template <typename TB, typename TS, typename TA, bool VAR>
__global__ void __launch_bounds__(256) mg_up(const TB* __restrict__ b, const TS* __restrict__ xcoarse,
                                             TS* __restrict__ x, int m, int mc, size_t ldb, size_t ldc, size_t ldx,
                                             const TA* __restrict__ st, TA omega, int nu1, int nu2, int tiles_x) {
  __shared__ TA sb[UWX * UWY], sx0[UWX * UWY], sx1[UWX * UWY], sxc[UCX * UCY];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int tile = blockIdx.x, blk = blockIdx.y;
  const int X0 = (tile % tiles_x) * UX, Y0 = (tile / tiles_x) * UY;
  const int H = nu1 + nu2 - 1;
  const int WX = UX + 2 * H, WY = UY + 2 * H;
  const int fi0 = X0 - H, fj0 = Y0 - H;
  const TB* bb = b + (size_t)blk * ldb;
  SG_WLOOP(WX, WY) {
    const int t = lj * WX + li, i = fi0 + li, j = fj0 + lj;
    TA v = 0, xv = 0;
    if (i >= 0 && i < m && j >= 0 && j < m) {
      v = ld_as<TA>(bb + (size_t)i + (size_t)j * m);
      const TA* sp = VAR ? st + 9 * ((size_t)i + (size_t)j * m) : nullptr;
      xv = omega * dinv_at<TA, VAR>(sp) * v;
    }
    sb[t] = v;
    sx0[t] = xv;
  }
  // coarse values covering fine [X0 - nu2, X0 + UX + nu2)
  const int ci0 = ((X0 - nu2) >> 1) - 1, cj0 = ((Y0 - nu2) >> 1) - 1;   // arithmetic shift = floor
  const int CWX = (UX + 2 * nu2) / 2 + 3, CWY = (UY + 2 * nu2) / 2 + 3;
  const TS* xcb = xcoarse + (size_t)blk * ldc;
  SG_WLOOP(CWX, CWY) {
    const int I = ci0 + li, J = cj0 + lj;
    sxc[lj * CWX + li] = (I >= 0 && I < mc && J >= 0 && J < mc) ? ld_as<TA>(xcb + (size_t)I + (size_t)J * mc) : TA(0);
  }
  __syncthreads();
  TA* xc = sx0;
  TA* xn = sx1;
  for (int s = 2; s <= nu1; ++s) {
    const int lo = s - 1;
    SG_WLOOP(WX, WY) {
      const int t = lj * WX + li, i = fi0 + li, j = fj0 + lj;
      TA v = 0;
      if (li >= lo && li < WX - lo && lj >= lo && lj < WY - lo && i >= 0 && i < m && j >= 0 && j < m) {
        const TA* sp = VAR ? st + 9 * ((size_t)i + (size_t)j * m) : nullptr;
        v = xc[t] + omega * dinv_at<TA, VAR>(sp) * (sb[t] - apply_pt<TA, VAR>(xc, WX, li, lj, sp));
      }
      xn[t] = v;
    }
    __syncthreads();
    TA* tmp = xc; xc = xn; xn = tmp;
  }
  {
    // coarse-grid correction on fine [X0 - nu2, X0 + UX + nu2): fine interior i <-> vertex i + 1;
    // an even vertex sits on a coarse vertex, an odd one between two (weights 1/2)
    const int lo = nu1 - 1;
    SG_WLOOP(WX, WY) {
      const int t = lj * WX + li, i = fi0 + li, j = fj0 + lj;
      if (li >= lo && li < WX - lo && lj >= lo && lj < WY - lo && i >= 0 && i < m && j >= 0 && j < m) {
        TA corr;
        const int ix = (i & 1) ? ((i - 1) >> 1) : ((i >> 1) - 1);
        const int iy = (j & 1) ? ((j - 1) >> 1) : ((j >> 1) - 1);
        const TA* c0 = sxc + (iy - cj0) * CWX + (ix - ci0);
        if (i & 1) {
          if (j & 1) corr = c0[0];
          else corr = TA(0.5) * (c0[0] + c0[CWX]);
        } else {
          if (j & 1) corr = TA(0.5) * (c0[0] + c0[1]);
          else corr = TA(0.25) * ((c0[0] + c0[1]) + (c0[CWX] + c0[CWX + 1]));
        }
        xc[t] += corr;
      }
    }
  }
  __syncthreads();
  for (int s = 1; s <= nu2; ++s) {
    const int lo = nu1 - 1 + s;
    SG_WLOOP(WX, WY) {
      const int t = lj * WX + li, i = fi0 + li, j = fj0 + lj;
      TA v = 0;
      if (li >= lo && li < WX - lo && lj >= lo && lj < WY - lo && i >= 0 && i < m && j >= 0 && j < m) {
        const TA* sp = VAR ? st + 9 * ((size_t)i + (size_t)j * m) : nullptr;
        v = xc[t] + omega * dinv_at<TA, VAR>(sp) * (sb[t] - apply_pt<TA, VAR>(xc, WX, li, lj, sp));
      }
      xn[t] = v;
    }
    __syncthreads();
    TA* tmp = xc; xc = xn; xn = tmp;
  }
  TS* xb = x + (size_t)blk * ldx;
  for (int oj = ty; oj < UY; oj += 8)
    for (int oi = tx; oi < UX; oi += 32) {
      const int i = X0 + oi, j = Y0 + oj;
      if (i < m && j < m) st_as<TS, TA>(xb + (size_t)i + (size_t)j * m, xc[(j - fj0) * WX + (i - fi0)]);
    }
}
// ---------------------------------------------------------------------------
// Constant-coefficient V(1,1) fast path (abar = 1, every level the Q1 stencil).
// With c = omega / (8/3) and A = 3 I - S9 / 3 (S9 = 3 x 3 box sum):
//   down:  b_c = P^T (b - A c b) = (1 - 3c) (r3 (x) r3) b + (c/3) (r5 (x) r5) b,
//          r3 = (1/2, 1, 1/2), r5 = r3 * (1,1,1) = (1/2, 3/2, 2, 3/2, 1/2), taps
//          centred on the fine node 2I+1 that carries coarse node I;
//   up:    x = c b + e (e = P x_c), then one Jacobi step:
//          x' = (2c - 3c^2) b + (1 - 3c) e + S9 g,   g = (c^2/3) b + (c/3) e.
// Both are separable filters evaluated in shared memory (row pass, then column pass).
constexpr int DCX = 32, DCY = 8;                         // coarse outputs per mg_down_c11 CTA
constexpr int DWX = 2 * DCX + 3, DWY = 2 * DCY + 3;      // fine window (67 x 19)
constexpr int UOX = 64, UOY = 16;                        // fine outputs per mg_up_c11 CTA
constexpr int UGX = UOX + 2, UGY = UOY + 2;              // g window (halo 1)
constexpr int UCWX = UOX / 2 + 3, UCWY = UOY / 2 + 3;    // coarse window

template <typename TB, typename TS, typename TA>
__global__ void __launch_bounds__(256) mg_down_c11(const TB* __restrict__ b, TS* __restrict__ bc, int m, int mc,
                                                   size_t ldb, size_t ldc, TA c, int tiles_x) {
  __shared__ TA sw[DWY][DWX];
  __shared__ TA h3[DWY][DCX], h5[DWY][DCX];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int tile = blockIdx.x, blk = blockIdx.y;
  const int I0 = (tile % tiles_x) * DCX, J0 = (tile / tiles_x) * DCY;
  const int fi0 = 2 * I0 - 1, fj0 = 2 * J0 - 1;        // window (0,0) = fine node 2 I0 + 1 - 2
  const TB* bb = b + (size_t)blk * ldb;
  for (int lj = ty; lj < DWY; lj += 8)
    for (int li = tx; li < DWX; li += 32) {
      const int i = fi0 + li, j = fj0 + lj;
      sw[lj][li] = (i >= 0 && i < m && j >= 0 && j < m) ? ld_as<TA>(bb + (size_t)i + (size_t)j * m) : TA(0);
    }
  __syncthreads();
  // row pass at the coarse x positions: fine 2I+1 is window column 2(I - I0) + 2
  for (int lj = ty; lj < DWY; lj += 8) {
    const TA* r = &sw[lj][2 * tx];
    const TA s3 = TA(0.5) * (r[1] + r[3]) + r[2];
    const TA s5 = TA(0.5) * (r[0] + r[4]) + TA(1.5) * (r[1] + r[3]) + TA(2) * r[2];
    h3[lj][tx] = s3;
    h5[lj][tx] = s5;
  }
  __syncthreads();
  const TA a3 = TA(1) - TA(3) * c, a5 = c / TA(3);
  {
    const int I = I0 + tx, J = J0 + ty;
    if (I < mc && J < mc) {
      const int lj = 2 * ty;                              // rows 2ty .. 2ty+4 centred on 2ty+2
      const TA v3 = TA(0.5) * (h3[lj + 1][tx] + h3[lj + 3][tx]) + h3[lj + 2][tx];
      const TA v5 = TA(0.5) * (h5[lj][tx] + h5[lj + 4][tx]) + TA(1.5) * (h5[lj + 1][tx] + h5[lj + 3][tx]) +
                    TA(2) * h5[lj + 2][tx];
      st_as<TS, TA>(bc + (size_t)blk * ldc + (size_t)I + (size_t)J * mc, a3 * v3 + a5 * v5);
    }
  }
}

template <typename TB, typename TS, typename TA>
__global__ void __launch_bounds__(256) mg_up_c11(const TB* __restrict__ b, const TS* __restrict__ xcoarse,
                                                 TS* __restrict__ x, int m, int mc, size_t ldb, size_t ldc, size_t ldx,
                                                 TA c, int tiles_x) {
  __shared__ TA sg[UGY][UGX];        // g on the output tile plus halo 1
  __shared__ TA sh[UGY][UOX];        // row sums of g
  __shared__ TA sbe[UOY][UOX];       // (2c - 3c^2) b + (1 - 3c) e on the output tile
  __shared__ TA sxc[UCWY][UCWX];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int tile = blockIdx.x, blk = blockIdx.y;
  const int X0 = (tile % tiles_x) * UOX, Y0 = (tile / tiles_x) * UOY;
  const int ci0 = (X0 >> 1) - 2, cj0 = (Y0 >> 1) - 2;   // coarse window origin
  const TS* xcb = xcoarse + (size_t)blk * ldc;
  for (int lj = ty; lj < UCWY; lj += 8)
    for (int li = tx; li < UCWX; li += 32) {
      const int I = ci0 + li, J = cj0 + lj;
      sxc[lj][li] = (I >= 0 && I < mc && J >= 0 && J < mc) ? ld_as<TA>(xcb + (size_t)I + (size_t)J * mc) : TA(0);
    }
  __syncthreads();
  const TB* bb = b + (size_t)blk * ldb;
  const TA cg_b = c * c / TA(3), cg_e = c / TA(3);
  const TA cb = TA(2) * c - TA(3) * c * c, ce = TA(1) - TA(3) * c;
  for (int lj = ty; lj < UGY; lj += 8)
    for (int li = tx; li < UGX; li += 32) {
      const int i = X0 - 1 + li, j = Y0 - 1 + lj;
      TA g = 0;
      if (i >= 0 && i < m && j >= 0 && j < m) {
        const TA bv = ld_as<TA>(bb + (size_t)i + (size_t)j * m);
        // e = P x_c at fine interior (i, j): odd index on a coarse node, even between two
        const int ix = (i & 1) ? ((i - 1) >> 1) : ((i >> 1) - 1);
        const int iy = (j & 1) ? ((j - 1) >> 1) : ((j >> 1) - 1);
        const TA* c0 = &sxc[iy - cj0][ix - ci0];
        TA e;
        if (i & 1) e = (j & 1) ? c0[0] : TA(0.5) * (c0[0] + c0[UCWX]);
        else e = (j & 1) ? TA(0.5) * (c0[0] + c0[1]) : TA(0.25) * ((c0[0] + c0[1]) + (c0[UCWX] + c0[UCWX + 1]));
        g = cg_b * bv + cg_e * e;
        if (li >= 1 && li <= UOX && lj >= 1 && lj <= UOY) sbe[lj - 1][li - 1] = cb * bv + ce * e;
      }
      sg[lj][li] = g;
    }
  __syncthreads();
  for (int lj = ty; lj < UGY; lj += 8)
    for (int li = tx; li < UOX; li += 32) sh[lj][li] = (sg[lj][li] + sg[lj][li + 1]) + sg[lj][li + 2];
  __syncthreads();
  TS* xb = x + (size_t)blk * ldx;
  for (int oj = ty; oj < UOY; oj += 8)
    for (int oi = tx; oi < UOX; oi += 32) {
      const int i = X0 + oi, j = Y0 + oj;
      if (i < m && j < m) {
        const TA v = sbe[oj][oi] + ((sh[oj][oi] + sh[oj + 1][oi]) + sh[oj + 2][oi]);
        st_as<TS, TA>(xb + (size_t)i + (size_t)j * m, v);
      }
    }
}
#undef SG_WLOOP
}  // namespace
