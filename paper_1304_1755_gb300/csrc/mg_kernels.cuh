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
template <typename TB, typename TS, typename TA, bool VAR, typename TO = TS>
__global__ void __launch_bounds__(256) mg_up(const TB* __restrict__ b, const TS* __restrict__ xcoarse,
                                             TO* __restrict__ x, int m, int mc, size_t ldb, size_t ldc, size_t ldx,
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
  TO* xb = x + (size_t)blk * ldx;
  for (int oj = ty; oj < UY; oj += 8)
    for (int oi = tx; oi < UX; oi += 32) {
      const int i = X0 + oi, j = Y0 + oj;
      if (i < m && j < m) st_as<TO, TA>(xb + (size_t)i + (size_t)j * m, xc[(j - fj0) * WX + (i - fi0)]);
    }
}
#undef SG_WLOOP
}  // namespace
