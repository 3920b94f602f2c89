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
//   mg_down_tile / mg_up_tile  the same two level steps for the common case of a
//            constant mean coefficient and V(1,1), as separable filters on
//            shared-memory windows filled by cp.async (mg_tile.cuh).
// Arithmetic type TA is double for SG_F64 and float otherwise; storage TS is
// double, float or bf16 (bf16: FP32 accumulation, storage only).
#include <algorithm>
#include <mutex>
#include <string>

#include "sg_internal.h"
#include "mg_kernels.cuh"
#include "mg_tile.cuh"

namespace {
constexpr int NC0 = 33;                                  // levels with n <= NC0 run in mg_coarse

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

template <typename TB, typename TS, typename TA, bool VAR, typename TO = TS>
__global__ void __launch_bounds__(512) mg_coarse(const TB* __restrict__ b, TO* __restrict__ x, size_t ldb,
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
  for (int t = threadIdx.x; t < m0 * m0; t += blockDim.x) st_as<TO, TA>(x + (size_t)blk * ldx + t, sx[t]);
}

// ---------------------------------------------------------------------------
template <typename TA> const TA* stencil_ptr(const sg_ctx* h, int l);
template <> const double* stencil_ptr<double>(const sg_ctx* h, int l) { return h->lev[l].st64; }
template <> const float* stencil_ptr<float>(const sg_ctx* h, int l) { return h->lev[l].st32; }

template <typename TB, typename TS, typename TA>
int run_down(sg_ctx* h, int l, int nb, const TB* b, TS* bc, bool bguard = false) {
  const MGLevel &F = h->lev[l], &C = h->lev[l + 1];
  if (h->const_mean && h->nu1 == 1) {
    const int tx = (C.m + MD_TX - 1) / MD_TX, ty = (C.m + MD_TY - 1) / MD_TY;
    const TA c = (TA)(h->omega * 3.0 / 8.0);
    if (bguard)
      mg_down_tile<TB, TS, TA, true><<<dim3(tx * ty, nb), MT_THREADS, 0, h->stream>>>(b, bc, F.m, C.m, F.N, C.N, c, tx);
    else
      mg_down_tile<TB, TS, TA, false><<<dim3(tx * ty, nb), MT_THREADS, 0, h->stream>>>(b, bc, F.m, C.m, F.N, C.N, c, tx);
    SG_CUDA(h, cudaGetLastError());
    count_launch(h);
    return SG_OK;
  }
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

template <typename TB, typename TS, typename TA, typename TO = TS>
int run_up(sg_ctx* h, int l, int nb, const TB* b, const TS* xc, TO* x, bool bguard = false, bool cguard = false,
           unsigned* zmax = nullptr) {
  const MGLevel &F = h->lev[l], &C = h->lev[l + 1];
  if (h->const_mean && h->nu1 == 1 && h->nu2 == 1) {
    constexpr int FY = mu_fy<TB, TS, TA>();
    const int tx = (F.m + MU_FX - 1) / MU_FX, ty = (F.m + FY - 1) / FY;
    const dim3 grid(tx * ty, nb);
    const TA c = (TA)(h->omega * 3.0 / 8.0);
    if (bguard && cguard)
      mg_up_tile<TB, TS, TA, TO, true, true><<<grid, MT_THREADS, 0, h->stream>>>(b, xc, x, F.m, C.m, F.N, C.N, F.N, c, tx,
                                                                                zmax);
    else if (cguard)
      mg_up_tile<TB, TS, TA, TO, false, true><<<grid, MT_THREADS, 0, h->stream>>>(b, xc, x, F.m, C.m, F.N, C.N, F.N, c,
                                                                                 tx, zmax);
    else
      mg_up_tile<TB, TS, TA, TO, false, false><<<grid, MT_THREADS, 0, h->stream>>>(b, xc, x, F.m, C.m, F.N, C.N, F.N, c,
                                                                                  tx, zmax);
    SG_CUDA(h, cudaGetLastError());
    count_launch(h);
    return SG_OK;
  }
  const int tx = (F.m + UX - 1) / UX, ty = (F.m + UY - 1) / UY;
  dim3 grid(tx * ty, nb);
  if (h->const_mean)
    mg_up<TB, TS, TA, false, TO><<<grid, 256, 0, h->stream>>>(b, xc, x, F.m, C.m, F.N, C.N, F.N, nullptr, (TA)h->omega,
                                                          h->nu1, h->nu2, tx);
  else
    mg_up<TB, TS, TA, true, TO><<<grid, 256, 0, h->stream>>>(b, xc, x, F.m, C.m, F.N, C.N, F.N, stencil_ptr<TA>(h, l),
                                                         (TA)h->omega, h->nu1, h->nu2, tx);
  SG_CUDA(h, cudaGetLastError());
  count_launch(h);
  return SG_OK;
}

template <typename TB, typename TS, typename TA, typename TO = TS>
int run_coarse(sg_ctx* h, int nb, const TB* b, TO* x) {
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
    auto kern = mg_coarse<TB, TS, TA, false, TO>;
    if (smem > 48 * 1024) SG_CUDA(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<nb, 512, smem, h->stream>>>(b, x, ldb, ldb, L, (TA)h->omega, h->nu1, h->nu2);
  } else {
    auto kern = mg_coarse<TB, TS, TA, true, TO>;
    if (smem > 48 * 1024) SG_CUDA(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<nb, 512, smem, h->stream>>>(b, x, ldb, ldb, L, (TA)h->omega, h->nu1, h->nu2);
  }
  SG_CUDA(h, cudaGetLastError());
  count_launch(h);
  return SG_OK;
}

// bguard: B lies in a guarded buffer; lguard: the level buffers of W are guarded (the handle's
// workspace is, the static scratch of sg_vcycle_static is not).
// zmax: see mg_up_tile (only on the tile path with levels below the fine grid; the caller checks)
template <typename TB, typename TS, typename TA, typename TO = TS>
int vcycle_t(sg_ctx* h, int nb, const TB* B, TO* X, PrecWork& W, bool bguard = false, bool lguard = false,
             unsigned* zmax = nullptr) {
  int rc;
  const int lc = h->lc;
  // descend
  for (int l = 0; l < lc; ++l) {
    if (l == 0) rc = run_down<TB, TS, TA>(h, 0, nb, B, (TS*)W.b[1], bguard);
    else rc = run_down<TS, TS, TA>(h, l, nb, (const TS*)W.b[l], (TS*)W.b[l + 1], lguard);
    if (rc) return rc;
  }
  if (lc == 0) rc = run_coarse<TB, TS, TA, TO>(h, nb, B, X);
  else rc = run_coarse<TS, TS, TA>(h, nb, (const TS*)W.b[lc], (TS*)W.x[lc]);
  if (rc) return rc;
  for (int l = lc - 1; l >= 0; --l) {
    if (l == 0) rc = run_up<TB, TS, TA, TO>(h, 0, nb, B, (const TS*)W.x[1], X, bguard, lguard, zmax);
    else rc = run_up<TS, TS, TA>(h, l, nb, (const TS*)W.b[l], (const TS*)W.x[l + 1], (TS*)W.x[l], lguard, lguard);
    if (rc) return rc;
  }
  return SG_OK;
}

// Buffers that the tile loaders may over-fetch around: 256 bytes before and 4 KB after the data
// (more than the widest window row), so whole aligned 16-byte chunks never leave the allocation.
constexpr size_t GUARD_FRONT = 256, GUARD_BACK = 4096;
}  // namespace

void* sg_galloc(size_t bytes) {
  void* p = nullptr;
  if (cudaMalloc(&p, bytes + GUARD_FRONT + GUARD_BACK) != cudaSuccess) return nullptr;
  return (char*)p + GUARD_FRONT;
}
void sg_gfree(void* p) {
  if (p) cudaFree((char*)p - GUARD_FRONT);
}

int ensure_prec_work(sg_ctx* h, int mode) {
  const int prec = wprec_of(mode);
  PrecWork& W = h->work[prec];
  if (mode == SG_BF16Z && !W.T32) {
    int nqmax = 0;
    for (int q = 0; q <= h->p; ++q) nqmax = std::max(nqmax, h->lvl_off[q + 1] - h->lvl_off[q]);
    if (!(W.T32 = sg_galloc(sizeof(float) * (size_t)nqmax * h->Nx)))
      return sg_fail(h, SG_E_ALLOC, "alloc FP32 stage buffer");
  }
  if (W.ready) return SG_OK;
  const size_t es = prec_size(prec);
  int nqmax = 0;
  for (int q = 0; q <= h->p; ++q) nqmax = std::max(nqmax, h->lvl_off[q + 1] - h->lvl_off[q]);
  if (!(W.T = sg_galloc(es * (size_t)nqmax * h->Nx))) return sg_fail(h, SG_E_ALLOC, "alloc stage buffer");
  for (int l = 1; l < (h->elements == SG_P1 ? 1 : h->nlev); ++l) {   // the P1 cycle keeps its own levels
    const size_t bytes = es * (size_t)h->P * h->lev[l].N;
    if (!(W.b[l] = sg_galloc(bytes)) || !(W.x[l] = sg_galloc(bytes)))
      return sg_fail(h, SG_E_ALLOC, "alloc multigrid level");
  }
  W.ready = true;
  return SG_OK;
}

int vcycle_run(sg_ctx* h, int prec, int nb, const void* B, int bprec, void* X, bool bguard, unsigned* zmax) {
  if (nb <= 0) return SG_OK;
  if (nb > h->P) return sg_fail(h, SG_E_ARG, "vcycle: more blocks than the workspace holds");
  if (h->elements == SG_P1) {
    if (prec != SG_F64 || bprec != SG_F64) return sg_fail(h, SG_E_ARG, "P1 elements: FP64 V-cycles only");
    return vcycle_p1(h, nb, (const double*)B, h->Nx, (double*)X, h->Nx);
  }
  int rc = ensure_prec_work(h, prec);
  if (rc) return rc;
  PrecWork& W = h->work[wprec_of(prec)];
  if (prec == SG_BF16Z) {                 // BF16 levels, FP32 output
    if (bprec == SG_F64)
      return vcycle_t<double, bf16, float, float>(h, nb, (const double*)B, (float*)X, W, bguard, true, zmax);
    if (bprec == SG_F32)
      return vcycle_t<float, bf16, float, float>(h, nb, (const float*)B, (float*)X, W, bguard, true, zmax);
    return vcycle_t<bf16, bf16, float, float>(h, nb, (const bf16*)B, (float*)X, W, bguard, true, zmax);
  }
  if (prec == SG_F64) {
    if (bprec != SG_F64) return sg_fail(h, SG_E_ARG, "vcycle: FP64 cycle needs FP64 input");
    return vcycle_t<double, double, double>(h, nb, (const double*)B, (double*)X, W, bguard, true);
  }
  if (prec == SG_F32) {
    if (bprec == SG_F64) return vcycle_t<double, float, float>(h, nb, (const double*)B, (float*)X, W, bguard, true, zmax);
    return vcycle_t<float, float, float>(h, nb, (const float*)B, (float*)X, W, bguard, true, zmax);
  }
  if (bprec == SG_F64) return vcycle_t<double, bf16, float>(h, nb, (const double*)B, (bf16*)X, W, bguard, true);
  if (bprec == SG_F32) return vcycle_t<float, bf16, float>(h, nb, (const float*)B, (bf16*)X, W, bguard, true);
  return vcycle_t<bf16, bf16, float>(h, nb, (const bf16*)B, (bf16*)X, W, bguard, true);
}

// A preconditioner application is a fixed sequence of about ten launches per degree
// stage (many on tiny coarse grids), so on a non-default stream it is captured once
// per operand set into a CUDA graph and replayed; the cache key is (R, Z, rprec,
// prec, kind, the block-maxima output).  Nested capture by the caller falls back to direct launches.
template <class Body>
int run_graphed(sg_ctx* h, const void* R, const void* Z, int rprec, int prec, int kind, Body&& body,
                const void* zmax = nullptr) {
  int rc = ensure_prec_work(h, prec);
  if (rc) return rc;
  if (h->stream == nullptr) return body();
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  SG_CUDA(h, cudaStreamIsCapturing(h->stream, &cs));
  if (cs != cudaStreamCaptureStatusNone) return body();
  const auto key = std::make_tuple(R, Z, rprec, prec, kind, zmax);
  auto it = h->graphs.find(key);
  if (it == h->graphs.end()) {
    if (h->graphs.size() >= 512) {
      for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second.exec);
      h->graphs.clear();
    }
    const long long before = h->tr.launches[h->phase];
    SG_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    rc = body();
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(h->stream, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (ec != cudaSuccess) return sg_fail(h, SG_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) return sg_fail(h, SG_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
    it = h->graphs.emplace(key, sg_ctx::GraphEntry{ex, h->tr.launches[h->phase] - before}).first;
  } else {
    count_launch(h, (int)it->second.kernels);
  }
  SG_CUDA(h, cudaGraphLaunch(it->second.exec, h->stream));
  return SG_OK;
}

// B_T^{-1} (Sec. 4.2): degree levels q are dependent stages; the n_q diagonal
// blocks of one stage are independent and cycled together.
static int precond_blocktri_direct(sg_ctx* h, int rprec, const void* R, void* Z, int prec, int transpose,
                                   unsigned* zmax) {
  int rc;
  if (zmax) SG_CUDA(h, cudaMemsetAsync(zmax, 0, sizeof(unsigned) * h->P, h->stream));
  // storage of Z, of the work buffers and of the stage right-hand side T (FP32 for SG_BF16Z: the
  // levels stay BF16, the vectors the Krylov method sees are FP32)
  const int zp = zprec_of(prec), wp = wprec_of(prec), tp = prec == SG_BF16Z ? SG_F32 : wp;
  const size_t es = prec_size(zp), rs = prec_size(rprec);
  const int arith = prec == SG_F64 ? SG_F64 : SG_F32;
  for (int s = 0; s <= h->p; ++s) {
    const int q = transpose ? h->p - s : s;
    const int r0 = h->lvl_off[q], nq = h->lvl_off[q + 1] - r0;
    char* Zq = (char*)Z + es * (size_t)r0 * h->Nx;
    if (s == 0) {
      rc = vcycle_run(h, prec, nq, (const char*)R + rs * (size_t)r0 * h->Nx, rprec, Zq, false, zmax ? zmax + r0 : nullptr);
    } else {
      // T_q = R_q - sum over the couplings to the previous stage of G_k(i,j) K_k Z_j
      void* T = prec == SG_BF16Z ? h->work[wp].T32 : h->work[wp].T;
      rc = launch_apply(h, transpose ? 2 : 1, zp, Z, 0, tp, T, 0, rprec, R, 0, r0, nq, r0, 0, arith);
      if (rc) return rc;
      rc = vcycle_run(h, prec, nq, T, tp, Zq, true, zmax ? zmax + r0 : nullptr);
    }
    if (rc) return rc;
  }
  return SG_OK;
}

int precond_blocktri(sg_ctx* h, int rprec, const void* R, void* Z, int prec, int transpose) {
  if (prec == SG_F64 && rprec != SG_F64) return sg_fail(h, SG_E_ARG, "blocktri: FP64 sweep needs FP64 input");
  // the output's block maxima come out of the level-0 up kernels when every stage takes that path
  // (constant mean, V(1,1), a level below the fine grid, FP32 output)
  unsigned* zmax = h->zmax_out && zprec_of(prec) == SG_F32 && h->elements == SG_Q1 && h->const_mean &&
                           h->nu1 == 1 && h->nu2 == 1 && h->lc > 0
                       ? h->zmax_out
                       : nullptr;
  const int rc = run_graphed(
      h, R, Z, rprec, prec, transpose ? 2 : 1,
      [&] { return precond_blocktri_direct(h, rprec, R, Z, prec, transpose, zmax); }, zmax);
  h->zmax_done = rc == SG_OK && zmax;
  return rc;
}

// B_S^{-1} (Sec. 4.2): B_S = B_T diag(A)^{-1} B_T^T, applied as a lower sweep, the exact
// diagonal blocks K_0 (one stencil pass) and an upper sweep.
int precond_blocksym(sg_ctx* h, int rprec, const void* R, void* Z, int prec) {
  if (prec == SG_F64 && rprec != SG_F64) return sg_fail(h, SG_E_ARG, "blocksym: FP64 sweep needs FP64 input");
  const int zp = zprec_of(prec);
  int rc = ensure_prec_work(h, prec);
  if (rc) return rc;
  PrecWork& W = h->work[wprec_of(prec)];
  const size_t N = h->Nx * (size_t)h->P;
  const int sprec = prec == SG_F64 ? SG_F64 : SG_F32;
  if (!W.S1 || W.s1_prec != zp) {
    cudaFree(W.S1);
    cudaFree(W.S2);
    W.S1 = W.S2 = nullptr;
    if (cudaMalloc(&W.S1, prec_size(zp) * N) != cudaSuccess || cudaMalloc(&W.S2, prec_size(sprec) * N) != cudaSuccess)
      return sg_fail(h, SG_E_ALLOC, "alloc symmetric sweep buffers");
    W.s1_prec = zp;
  }
  if ((rc = precond_blocktri(h, rprec, R, W.S1, prec, 0))) return rc;
  if ((rc = launch_apply(h, 4, zp, W.S1, 0, sprec, W.S2, 0, SG_F64, nullptr, 0, 0, h->P, 0, 0, sprec))) return rc;
  return precond_blocktri(h, sprec, W.S2, Z, prec, 1);
}

// B_S^{-1} in the recursive 2 x 2 form of Sec. 4.2 (FP64).  rec(q, R, Z): R holds the blocks of
// degrees 0..q (block-contiguous from block 0), Z receives B_q^{-1} R in the same blocks.  Only degrees
// q - 1 and q couple (G_k, k >= 1, changes one index by one), so W y_low reads the degree q - 1 blocks of
// y_low and W^T y_q changes only the degree q - 1 rows of R_low; those rows go to a per-depth copy of
// R_low.  Every step is an existing launch: the coupling tables' R - AX epilogue and the batched cycle.
static int blocksym_rec(sg_ctx* h, int q, const double* R, double* Z) {
  int rc;
  const size_t Nx = h->Nx;
  if (q == 0) return vcycle_run(h, SG_F64, 1, R, SG_F64, Z, false);
  const int lo = h->lvl_off[q], nq = h->lvl_off[q + 1] - lo, l1 = h->lvl_off[q - 1], n1 = lo - l1;
  if ((rc = blocksym_rec(h, q - 1, R, Z))) return rc;                       // y_low
  double* T = (double*)h->work[SG_F64].T;                                     // R_q - W y_low
  if ((rc = launch_apply(h, 1, SG_F64, Z, 0, SG_F64, T, 0, SG_F64, R, 0, lo, nq, lo, 0, SG_F64))) return rc;
  if ((rc = vcycle_run(h, SG_F64, nq, T, SG_F64, Z + (size_t)lo * Nx, true))) return rc;   // y_q
  double* Rl = h->bsr + h->bsr_off[q];                                        // R_low - W^T y_q
  if (l1 > 0) SG_CUDA(h, cudaMemcpyAsync(Rl, R, sizeof(double) * Nx * l1, cudaMemcpyDeviceToDevice, h->stream));
  if ((rc = launch_apply(h, 2, SG_F64, Z, 0, SG_F64, Rl + (size_t)l1 * Nx, 0, SG_F64, R, 0, l1, n1, l1, 0, SG_F64)))
    return rc;
  return blocksym_rec(h, q - 1, Rl, Z);                                       // z_low
}

int precond_blocksym_rec(sg_ctx* h, int rprec, const void* R, void* Z, int prec) {
  if (rprec != SG_F64 || prec != SG_F64) return sg_fail(h, SG_E_ARG, "recursive B_S: FP64 only");
  int rc = ensure_prec_work(h, SG_F64);
  if (rc) return rc;
  if (!h->bsr && h->p > 0) {               // per depth q >= 1: a copy of the blocks of degrees < q
    size_t tot = 0;
    for (int q = 1; q <= h->p; ++q) h->bsr_off[q] = tot, tot += (size_t)h->lvl_off[q] * h->Nx;
    if (cudaMalloc(&h->bsr, sizeof(double) * tot) != cudaSuccess) return sg_fail(h, SG_E_ALLOC, "alloc recursive B_S work");
  }
  return run_graphed(h, R, Z, SG_F64, SG_F64, 3, [&] { return blocksym_rec(h, h->p, (const double*)R, (double*)Z); });
}

// B_D^{-1} (Sec. 4.1): one V-cycle on every PC block.
int precond_blockdiag(sg_ctx* h, int rprec, const void* R, void* Z, int prec) {
  if (prec == SG_F64 && rprec != SG_F64) return sg_fail(h, SG_E_ARG, "blockdiag: FP64 cycle needs FP64 input");
  return run_graphed(h, R, Z, rprec, prec, 0, [&] { return vcycle_run(h, prec, h->P, R, rprec, Z); });
}

// ---------------------------------------------------------------------------
// sg_vcycle_static: the V-cycle of sg_vcycle with its coarse-level buffers taken from
// a fixed array compiled into the library instead of the handle's lazily allocated
// workspace, so a call never allocates device memory.
//
// Layout inside the array: for l = 1 .. lc (the levels below the fine grid that the
// level kernels touch), the right-hand sides b_l then the solutions x_l, each nblocks x
// N_l values of the cycle's storage type, every region starting on a 256-byte boundary.
// Levels coarser than lc live in the single-CTA kernel's shared memory and need no storage.
// Every value a call reads from the array was written earlier in the same call (the
// restriction writes all of b_{l+1}, the coarse kernel all of x_lc, the prolongation
// all of x_l), so nothing has to be cleared between calls.
namespace {
constexpr size_t VCYCLE_SCRATCH_BYTES = size_t(32) << 20;   // 32 MiB
__device__ __align__(256) unsigned char g_vcycle_scratch[VCYCLE_SCRATCH_BYTES];

constexpr int SCRATCH_MAX_DEVICES = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[SCRATCH_MAX_DEVICES] = {};

// Looks up (once per device, with that device current) the device address of the array.
int scratch_address(sg_ctx* h, unsigned char** out) {
  int dev = 0;
  SG_CUDA(h, cudaGetDevice(&dev));
  if (dev < 0 || dev >= SCRATCH_MAX_DEVICES) return sg_fail(h, SG_E_ARG, "sg_vcycle_static: device index out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_vcycle_scratch);
    if (e != cudaSuccess || !p)
      return sg_fail(h, SG_E_CUDA, std::string("sg_vcycle_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = (unsigned char*)g_scratch_addr[dev];
  return SG_OK;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

size_t static_scratch_bytes(const sg_ctx* h, int nblocks, int prec) {
  size_t need = 0;
  for (int l = 1; l <= h->lc; ++l) need += 2 * align256(prec_size(prec) * (size_t)nblocks * h->lev[l].N);
  return need;
}
}  // namespace

extern "C" int sg_vcycle_static(sg_handle h, const double* B, void* X, int nblocks, int prec) {
  if (!h || !B || !X || prec < 0 || prec > 2 || nblocks < 0 || nblocks > h->P)
    return h ? sg_fail(h, SG_E_ARG, "sg_vcycle_static: bad argument") : SG_E_ARG;
  if (const int rcd = sg_check_device(h, "sg_vcycle_static")) return rcd;   // the array's address is per device
  if (h->elements != SG_Q1) return sg_fail(h, SG_E_ARG, "sg_vcycle_static: Q1 elements only");
  if (nblocks == 0) return SG_OK;
  const size_t need = static_scratch_bytes(h, nblocks, prec);
  if (need > VCYCLE_SCRATCH_BYTES)
    return sg_fail(h, SG_E_ARG, "sg_vcycle_static: " + std::to_string(nblocks) + " blocks need " +
                                    std::to_string(need) + " bytes of scratch, the static array holds " +
                                    std::to_string(VCYCLE_SCRATCH_BYTES) + "; use sg_vcycle or fewer blocks");
  unsigned char* base = nullptr;
  int rc = scratch_address(h, &base);
  if (rc) return rc;
  PrecWork W;                                     // views into the array; nothing is allocated
  size_t off = 0;
  for (int l = 1; l <= h->lc; ++l) {
    const size_t bytes = align256(prec_size(prec) * (size_t)nblocks * h->lev[l].N);
    W.b[l] = base + off;
    off += bytes;
    W.x[l] = base + off;
    off += bytes;
  }
  if (prec == SG_F64) return vcycle_t<double, double, double>(h, nblocks, B, (double*)X, W);
  if (prec == SG_F32) return vcycle_t<double, float, float>(h, nblocks, B, (float*)X, W);
  return vcycle_t<double, bf16, float>(h, nblocks, B, (bf16*)X, W);
}
