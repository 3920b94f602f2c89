// Geometric multigrid V-cycle on the mean operator K_0 and the two block
// preconditioners built on it (Sec. 4.1 B_D, Sec. 4.2 B_T).
//
// V(nu1, nu2) cycle from a zero initial guess, damped Jacobi smoothing, bilinear
// prolongation P, restriction P^T, Galerkin coarse operators (for abar = 1 every
// level is the Q1 stencil 8/3, -1/3), coarsest grid (one unknown) solved in FP64.
// All blocks of a call are cycled together (the diagonal blocks are independent).
//
// Kernels
//   mg_down  level l -> l+1: pre-smoothing from zero, residual and restriction
//            fused in shared memory; reads b_l once, writes b_{l+1}.  The
//            pre-smoothed x_l is not stored.
//   mg_up    level l+1 -> l: recomputes the pre-smoothed x_l from b_l,
//            adds P x_{l+1}, post-smooths; reads b_l and x_{l+1}, writes x_l.
//   mg_coarse one CTA per block runs every level with n_l <= 33 (down, coarsest
//            solve, up) in shared memory.
// Arithmetic type TA is double for SG_F64 and float otherwise; storage TS is
// double, float or bf16 (bf16: FP32 accumulation, storage only).
#include <algorithm>

#include "sg_internal.h"

namespace {
constexpr int MAXNU = 4;
constexpr int CT = 16;                                   // coarse tile of mg_down
constexpr int DW = 2 * CT + 1 + 2 * MAXNU;               // its fine window
constexpr int UX = 32, UY = 16;                          // fine tile of mg_up
constexpr int UH = 2 * MAXNU - 1;
constexpr int UWX = UX + 2 * UH, UWY = UY + 2 * UH;
constexpr int UCX = (UX + 2 * MAXNU) / 2 + 3, UCY = (UY + 2 * MAXNU) / 2 + 3;
constexpr int NC0 = 33;                                  // levels with n <= NC0 run in mg_coarse

template <typename TA> struct Q1 {
  static __device__ __forceinline__ TA diag() { return TA(8) / TA(3); }
};

// A x at window point (li, lj) of a row-major window of width w.
template <typename TA, bool VAR>
__device__ __forceinline__ TA apply_pt(const TA* x, int w, int li, int lj, const TA* st) {
  const TA* r0 = x + (lj - 1) * w + li;
  const TA* r1 = r0 + w;
  const TA* r2 = r1 + w;
  if (VAR) {
    return st[0] * r0[-1] + st[1] * r0[0] + st[2] * r0[1] + st[3] * r1[-1] + st[4] * r1[0] + st[5] * r1[1] +
           st[6] * r2[-1] + st[7] * r2[0] + st[8] * r2[1];
  }
  const TA s9 = (r0[-1] + r0[0] + r0[1]) + (r1[-1] + r1[0] + r1[1]) + (r2[-1] + r2[0] + r2[1]);
  return TA(3) * r1[0] - s9 * (TA(1) / TA(3));
}

template <typename TA, bool VAR>
__device__ __forceinline__ TA dinv_at(const TA* st) {
  if (VAR) return TA(1) / st[4];
  return TA(3) / TA(8);
}

// ---------------------------------------------------------------------------
template <typename TB, typename TS, typename TA, bool VAR>
__global__ void __launch_bounds__(256) mg_down(const TB* __restrict__ b, TS* __restrict__ bc, int m, int mc,
                                               size_t ldb, size_t ldc, const TA* __restrict__ st, TA omega,
                                               int nu1, int tiles_x) {
  __shared__ TA sb[DW * DW], sx0[DW * DW], sx1[DW * DW];
  const int tile = blockIdx.x, blk = blockIdx.y;
  const int I0 = (tile % tiles_x) * CT, J0 = (tile / tiles_x) * CT;
  const int W = 2 * CT + 1 + 2 * nu1;
  const int fi0 = 2 * I0 - nu1, fj0 = 2 * J0 - nu1;     // fine interior index of window (0,0)
  const TB* bb = b + (size_t)blk * ldb;
  for (int t = threadIdx.x; t < W * W; t += blockDim.x) {
    const int li = t % W, lj = t / W, i = fi0 + li, j = fj0 + lj;
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
    for (int t = threadIdx.x; t < W * W; t += blockDim.x) {
      const int li = t % W, lj = t / W, i = fi0 + li, j = fj0 + lj;
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
  // residual on the inner (2 CT + 1)^2 window, written over a second buffer
  {
    const int lo = nu1, hi = W - nu1;
    for (int t = threadIdx.x; t < W * W; t += blockDim.x) {
      const int li = t % W, lj = t / W, i = fi0 + li, j = fj0 + lj;
      TA r = 0;
      if (li >= lo && li < hi && lj >= lo && lj < hi && i >= 0 && i < m && j >= 0 && j < m) {
        const TA* sp = VAR ? st + 9 * ((size_t)i + (size_t)j * m) : nullptr;
        r = sb[t] - apply_pt<TA, VAR>(xc, W, li, lj, sp);
      }
      xn[t] = r;
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < CT * CT; t += blockDim.x) {
    const int I = I0 + t % CT, J = J0 + t / CT;
    if (I < mc && J < mc) {
      const int li = 2 * I - fi0, lj = 2 * J - fj0;        // window index of fine node 2I (weight 1/2)
      const TA* r0 = xn + lj * W + li;
      const TA* r1 = r0 + W;
      const TA* r2 = r1 + W;
      const TA v = TA(0.25) * (r0[0] + r0[2] + r2[0] + r2[2]) + TA(0.5) * (r0[1] + r1[0] + r1[2] + r2[1]) + r1[1];
      st_as<TS, TA>(bc + (size_t)blk * ldc + (size_t)I + (size_t)J * mc, v);
    }
  }
}

// ---------------------------------------------------------------------------
template <typename TB, typename TS, typename TA, bool VAR>
__global__ void __launch_bounds__(256) mg_up(const TB* __restrict__ b, const TS* __restrict__ xcoarse,
                                             TS* __restrict__ x, int m, int mc, size_t ldb, size_t ldc, size_t ldx,
                                             const TA* __restrict__ st, TA omega, int nu1, int nu2, int tiles_x) {
  __shared__ TA sb[UWX * UWY], sx0[UWX * UWY], sx1[UWX * UWY], sxc[UCX * UCY];
  const int tile = blockIdx.x, blk = blockIdx.y;
  const int X0 = (tile % tiles_x) * UX, Y0 = (tile / tiles_x) * UY;
  const int H = nu1 + nu2 - 1;
  const int WX = UX + 2 * H, WY = UY + 2 * H;
  const int fi0 = X0 - H, fj0 = Y0 - H;
  const TB* bb = b + (size_t)blk * ldb;
  for (int t = threadIdx.x; t < WX * WY; t += blockDim.x) {
    const int li = t % WX, lj = t / WX, i = fi0 + li, j = fj0 + lj;
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
  const int ci0 = ((X0 - nu2) >> 1) - 1, cj0 = ((Y0 - nu2) >> 1) - 1;  // arithmetic shift = floor
  const int CWX = (UX + 2 * nu2) / 2 + 3, CWY = (UY + 2 * nu2) / 2 + 3;
  const TS* xcb = xcoarse + (size_t)blk * ldc;
  for (int t = threadIdx.x; t < CWX * CWY; t += blockDim.x) {
    const int I = ci0 + t % CWX, J = cj0 + t / CWX;
    sxc[t] = (I >= 0 && I < mc && J >= 0 && J < mc) ? ld_as<TA>(xcb + (size_t)I + (size_t)J * mc) : TA(0);
  }
  __syncthreads();
  TA* xc = sx0;
  TA* xn = sx1;
  for (int s = 2; s <= nu1; ++s) {
    const int lo = s - 1;
    for (int t = threadIdx.x; t < WX * WY; t += blockDim.x) {
      const int li = t % WX, lj = t / WX, i = fi0 + li, j = fj0 + lj;
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
  // coarse-grid correction on fine [X0 - nu2, X0 + UX + nu2)
  {
    const int lo = nu1 - 1;
    for (int t = threadIdx.x; t < WX * WY; t += blockDim.x) {
      const int li = t % WX, lj = t / WX, i = fi0 + li, j = fj0 + lj;
      if (li >= lo && li < WX - lo && lj >= lo && lj < WY - lo && i >= 0 && i < m && j >= 0 && j < m) {
        // fine interior i <-> vertex i+1; even vertex sits on coarse vertex (i+1)/2 (interior (i-1)/2)
        TA px[2], py[2];
        int ix[2], iy[2], nx, ny;
        if (i & 1) { ix[0] = (i - 1) >> 1; px[0] = 1; nx = 1; }
        else { ix[0] = (i >> 1) - 1; ix[1] = i >> 1; px[0] = px[1] = TA(0.5); nx = 2; }
        if (j & 1) { iy[0] = (j - 1) >> 1; py[0] = 1; ny = 1; }
        else { iy[0] = (j >> 1) - 1; iy[1] = j >> 1; py[0] = py[1] = TA(0.5); ny = 2; }
        TA corr = 0;
        for (int a = 0; a < ny; ++a)
          for (int c = 0; c < nx; ++c) corr += py[a] * px[c] * sxc[(iy[a] - cj0) * CWX + (ix[c] - ci0)];
        xc[t] += corr;
      }
    }
  }
  __syncthreads();
  for (int s = 1; s <= nu2; ++s) {
    const int lo = nu1 - 1 + s;
    for (int t = threadIdx.x; t < WX * WY; t += blockDim.x) {
      const int li = t % WX, lj = t / WX, i = fi0 + li, j = fj0 + lj;
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
  for (int t = threadIdx.x; t < UX * UY; t += blockDim.x) {
    const int i = X0 + t % UX, j = Y0 + t / UX;
    if (i < m && j < m) st_as<TS, TA>(xb + (size_t)i + (size_t)j * m, xc[(j - fj0) * WX + (i - fi0)]);
  }
}

// ---------------------------------------------------------------------------
struct CoarseLevels {
  int nl;                 // number of levels handled
  int m[SG_MAX_LEVELS];
  int off[SG_MAX_LEVELS]; // offset of level arrays inside the b / x regions
  const void* st[SG_MAX_LEVELS];
};

template <typename TA, bool VAR>
__device__ void cg_smooth(const TA* b, TA* x, TA* tmp, int m, const TA* st, TA omega, bool from_zero) {
  // one damped-Jacobi step on an m x m grid held in shared memory
  if (from_zero) {
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) x[t] = omega * dinv_at<TA, VAR>(VAR ? st + 9 * t : nullptr) * b[t];
    __syncthreads();
    return;
  }
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    const int i = t % m, j = t / m;
    TA ax = 0;
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int ii = i + dx, jj = j + dy;
        if (ii < 0 || ii >= m || jj < 0 || jj >= m) continue;
        const TA c = VAR ? st[9 * t + (dy + 1) * 3 + (dx + 1)] : ((dx == 0 && dy == 0) ? TA(8) / TA(3) : TA(-1) / TA(3));
        ax += c * x[ii + jj * m];
      }
    tmp[t] = x[t] + omega * dinv_at<TA, VAR>(VAR ? st + 9 * t : nullptr) * (b[t] - ax);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) x[t] = tmp[t];
  __syncthreads();
}

template <typename TB, typename TS, typename TA, bool VAR>
__global__ void __launch_bounds__(512) mg_coarse(const TB* __restrict__ b, TS* __restrict__ x, size_t ldb,
                                                 size_t ldx, CoarseLevels L, TA omega, int nu1, int nu2) {
  extern __shared__ unsigned char smem_raw[];
  TA* sm = reinterpret_cast<TA*>(smem_raw);
  const int tot = L.off[L.nl - 1] + L.m[L.nl - 1] * L.m[L.nl - 1];
  TA* sb = sm;
  TA* sx = sm + tot;
  TA* tmp = sm + 2 * tot;
  const int blk = blockIdx.x;
  const int m0 = L.m[0];
  for (int t = threadIdx.x; t < m0 * m0; t += blockDim.x) sb[t] = ld_as<TA>(b + (size_t)blk * ldb + t);
  __syncthreads();
  for (int l = 0; l + 1 < L.nl; ++l) {
    const int m = L.m[l], mc = L.m[l + 1];
    TA *bl = sb + L.off[l], *xl = sx + L.off[l];
    const TA* st = (const TA*)L.st[l];
    cg_smooth<TA, VAR>(bl, xl, tmp, m, st, omega, true);
    for (int s = 1; s < nu1; ++s) cg_smooth<TA, VAR>(bl, xl, tmp, m, st, omega, false);
    // residual into tmp
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
      const int i = t % m, j = t / m;
      TA ax = 0;
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int ii = i + dx, jj = j + dy;
          if (ii < 0 || ii >= m || jj < 0 || jj >= m) continue;
          const TA c = VAR ? st[9 * t + (dy + 1) * 3 + (dx + 1)] : ((dx == 0 && dy == 0) ? TA(8) / TA(3) : TA(-1) / TA(3));
          ax += c * xl[ii + jj * m];
        }
      tmp[t] = bl[t] - ax;
    }
    __syncthreads();
    TA* bcl = sb + L.off[l + 1];
    for (int t = threadIdx.x; t < mc * mc; t += blockDim.x) {
      const int I = t % mc, J = t / mc;
      TA v = 0;
      for (int dy = 0; dy < 3; ++dy)
        for (int dx = 0; dx < 3; ++dx) {
          const TA w = (dx == 1 ? TA(1) : TA(0.5)) * (dy == 1 ? TA(1) : TA(0.5));
          v += w * tmp[(2 * I + dx) + (2 * J + dy) * m];
        }
      bcl[t] = v;
    }
    __syncthreads();
  }
  {
    // coarsest grid, solved exactly in FP64 (one unknown for n = 3; Jacobi-free direct division)
    const int l = L.nl - 1, m = L.m[l];
    const TA* st = (const TA*)L.st[l];
    if (m == 1 && threadIdx.x == 0) {
      const double d = VAR ? (double)st[4] : 8.0 / 3.0;
      sx[L.off[l]] = (TA)((double)sb[L.off[l]] / d);
    }
    __syncthreads();
  }
  for (int l = L.nl - 2; l >= 0; --l) {
    const int m = L.m[l], mc = L.m[l + 1];
    TA *bl = sb + L.off[l], *xl = sx + L.off[l];
    const TA* xcl = sx + L.off[l + 1];
    const TA* st = (const TA*)L.st[l];
    // recompute pre-smoothing (x_l was overwritten by nothing: still valid), add P x_c
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
      const int i = t % m, j = t / m;
      TA px[2], py[2];
      int ix[2], iy[2], nx, ny;
      if (i & 1) { ix[0] = (i - 1) >> 1; px[0] = 1; nx = 1; }
      else { ix[0] = (i >> 1) - 1; ix[1] = i >> 1; px[0] = px[1] = TA(0.5); nx = 2; }
      if (j & 1) { iy[0] = (j - 1) >> 1; py[0] = 1; ny = 1; }
      else { iy[0] = (j >> 1) - 1; iy[1] = j >> 1; py[0] = py[1] = TA(0.5); ny = 2; }
      TA corr = 0;
      for (int a = 0; a < ny; ++a)
        for (int c = 0; c < nx; ++c)
          if (ix[c] >= 0 && ix[c] < mc && iy[a] >= 0 && iy[a] < mc) corr += py[a] * px[c] * xcl[ix[c] + iy[a] * mc];
      xl[t] += corr;
    }
    __syncthreads();
    for (int s = 0; s < nu2; ++s) cg_smooth<TA, VAR>(bl, xl, tmp, m, st, omega, false);
  }
  for (int t = threadIdx.x; t < m0 * m0; t += blockDim.x) st_as<TS, TA>(x + (size_t)blk * ldx + t, sx[t]);
}

// ---------------------------------------------------------------------------
template <typename TA> const TA* stencil_ptr(const sg_ctx* h, int l);
template <> const double* stencil_ptr<double>(const sg_ctx* h, int l) { return h->lev[l].st64; }
template <> const float* stencil_ptr<float>(const sg_ctx* h, int l) { return h->lev[l].st32; }

template <typename TB, typename TS, typename TA>
int run_down(sg_ctx* h, int l, int nb, const TB* b, TS* bc) {
  const MGLevel &F = h->lev[l], &C = h->lev[l + 1];
  const int tiles_x = (C.m + CT - 1) / CT;
  dim3 grid(tiles_x * tiles_x, nb);
  if (h->const_mean)
    mg_down<TB, TS, TA, false><<<grid, 256, 0, h->stream>>>(b, bc, F.m, C.m, F.N, C.N, nullptr, (TA)h->omega, h->nu1, tiles_x);
  else
    mg_down<TB, TS, TA, true><<<grid, 256, 0, h->stream>>>(b, bc, F.m, C.m, F.N, C.N, stencil_ptr<TA>(h, l),
                                                            (TA)h->omega, h->nu1, tiles_x);
  SG_CUDA(h, cudaGetLastError());
  count_launch(h);
  return SG_OK;
}

template <typename TB, typename TS, typename TA>
int run_up(sg_ctx* h, int l, int nb, const TB* b, const TS* xc, TS* x) {
  const MGLevel &F = h->lev[l], &C = h->lev[l + 1];
  const int tx = (F.m + UX - 1) / UX, ty = (F.m + UY - 1) / UY;
  dim3 grid(tx * ty, nb);
  if (h->const_mean)
    mg_up<TB, TS, TA, false><<<grid, 256, 0, h->stream>>>(b, xc, x, F.m, C.m, F.N, C.N, F.N, nullptr, (TA)h->omega,
                                                          h->nu1, h->nu2, tx);
  else
    mg_up<TB, TS, TA, true><<<grid, 256, 0, h->stream>>>(b, xc, x, F.m, C.m, F.N, C.N, F.N, stencil_ptr<TA>(h, l),
                                                         (TA)h->omega, h->nu1, h->nu2, tx);
  SG_CUDA(h, cudaGetLastError());
  count_launch(h);
  return SG_OK;
}

template <typename TB, typename TS, typename TA>
int run_coarse(sg_ctx* h, int nb, const TB* b, TS* x) {
  CoarseLevels L{};
  L.nl = h->nlev - h->lc;
  int off = 0;
  for (int q = 0; q < L.nl; ++q) {
    const MGLevel& lv = h->lev[h->lc + q];
    L.m[q] = lv.m;
    L.off[q] = off;
    off += lv.m * lv.m;
    L.st[q] = stencil_ptr<TA>(h, h->lc + q);
  }
  const size_t smem = (size_t)(2 * off + L.m[0] * L.m[0]) * sizeof(TA);
  const size_t ldb = h->lev[h->lc].N;
  if (h->const_mean) {
    auto kern = mg_coarse<TB, TS, TA, false>;
    if (smem > 48 * 1024) SG_CUDA(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<nb, 512, smem, h->stream>>>(b, x, ldb, ldb, L, (TA)h->omega, h->nu1, h->nu2);
  } else {
    auto kern = mg_coarse<TB, TS, TA, true>;
    if (smem > 48 * 1024) SG_CUDA(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<nb, 512, smem, h->stream>>>(b, x, ldb, ldb, L, (TA)h->omega, h->nu1, h->nu2);
  }
  SG_CUDA(h, cudaGetLastError());
  count_launch(h);
  return SG_OK;
}

template <typename TB, typename TS, typename TA>
int vcycle_t(sg_ctx* h, int nb, const TB* B, TS* X, PrecWork& W) {
  int rc;
  const int lc = h->lc;
  // descend
  for (int l = 0; l < lc; ++l) {
    if (l == 0) rc = run_down<TB, TS, TA>(h, 0, nb, B, (TS*)W.b[1]);
    else rc = run_down<TS, TS, TA>(h, l, nb, (const TS*)W.b[l], (TS*)W.b[l + 1]);
    if (rc) return rc;
  }
  if (lc == 0) rc = run_coarse<TB, TS, TA>(h, nb, B, X);
  else rc = run_coarse<TS, TS, TA>(h, nb, (const TS*)W.b[lc], (TS*)W.x[lc]);
  if (rc) return rc;
  for (int l = lc - 1; l >= 0; --l) {
    if (l == 0) rc = run_up<TB, TS, TA>(h, 0, nb, B, (const TS*)W.x[1], X);
    else rc = run_up<TS, TS, TA>(h, l, nb, (const TS*)W.b[l], (const TS*)W.x[l + 1], (TS*)W.x[l]);
    if (rc) return rc;
  }
  return SG_OK;
}
}  // namespace

int ensure_prec_work(sg_ctx* h, int prec) {
  PrecWork& W = h->work[prec];
  if (W.ready) return SG_OK;
  const size_t es = prec_size(prec);
  int nqmax = 0;
  for (int q = 0; q <= h->p; ++q) nqmax = std::max(nqmax, h->lvl_off[q + 1] - h->lvl_off[q]);
  if (cudaMalloc(&W.T, es * (size_t)nqmax * h->Nx) != cudaSuccess) return sg_fail(h, SG_E_ALLOC, "alloc stage buffer");
  for (int l = 1; l < h->nlev; ++l) {
    const size_t bytes = es * (size_t)h->P * h->lev[l].N;
    if (cudaMalloc(&W.b[l], bytes) != cudaSuccess || cudaMalloc(&W.x[l], bytes) != cudaSuccess)
      return sg_fail(h, SG_E_ALLOC, "alloc multigrid level");
  }
  W.ready = true;
  return SG_OK;
}

int vcycle_run(sg_ctx* h, int prec, int nb, const void* B, int bprec, void* X) {
  if (nb <= 0) return SG_OK;
  if (nb > h->P) return sg_fail(h, SG_E_ARG, "vcycle: more blocks than the workspace holds");
  int rc = ensure_prec_work(h, prec);
  if (rc) return rc;
  PrecWork& W = h->work[prec];
  if (prec == SG_F64) {
    if (bprec != SG_F64) return sg_fail(h, SG_E_ARG, "vcycle: FP64 cycle needs FP64 input");
    return vcycle_t<double, double, double>(h, nb, (const double*)B, (double*)X, W);
  }
  if (prec == SG_F32) {
    if (bprec == SG_F64) return vcycle_t<double, float, float>(h, nb, (const double*)B, (float*)X, W);
    return vcycle_t<float, float, float>(h, nb, (const float*)B, (float*)X, W);
  }
  if (bprec == SG_F64) return vcycle_t<double, bf16, float>(h, nb, (const double*)B, (bf16*)X, W);
  return vcycle_t<bf16, bf16, float>(h, nb, (const bf16*)B, (bf16*)X, W);
}

// B_T^{-1} (Sec. 4.2): degree levels q are dependent stages; the n_q diagonal
// blocks of one stage are independent and cycled together.
int precond_blocktri(sg_ctx* h, const double* R, void* Z, int prec, int transpose) {
  int rc = ensure_prec_work(h, prec);
  if (rc) return rc;
  const size_t es = prec_size(prec);
  for (int s = 0; s <= h->p; ++s) {
    const int q = transpose ? h->p - s : s;
    const int r0 = h->lvl_off[q], nq = h->lvl_off[q + 1] - r0;
    char* Zq = (char*)Z + es * (size_t)r0 * h->Nx;
    if (s == 0) {
      rc = vcycle_run(h, prec, nq, R + (size_t)r0 * h->Nx, SG_F64, Zq);
    } else {
      // T_q = R_q - sum over the couplings to the previous stage of G_k(i,j) K_k Z_j
      rc = launch_apply(h, transpose ? 2 : 1, prec, Z, prec, h->work[prec].T, R, r0, nq, r0, 0, prec == SG_F64);
      if (rc) return rc;
      rc = vcycle_run(h, prec, nq, h->work[prec].T, prec, Zq);
    }
    if (rc) return rc;
  }
  return SG_OK;
}

// B_D^{-1} (Sec. 4.1): one V-cycle on every PC block.
int precond_blockdiag(sg_ctx* h, const double* R, void* Z, int prec) {
  return vcycle_run(h, prec, h->P, R, SG_F64, Z);
}
