// C-ABI entry points: set-up, operator, preconditioners and the Krylov drivers
// (Sec. 4.2: GMRES / flexible GMRES / GPCG[1] / PCG around B_T or B_D).
// The Krylov loops run on the host; every vector operation runs in this
// library's kernels and only scalars (Hessenberg columns, norms) cross to the host.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "df64.cuh"
#include "sg_internal.h"

namespace {
std::string g_setup_err;
std::mutex g_err_mu;

template <typename T>
int upload(sg_ctx* h, T** dst, const T* src, size_t count) {
  if (count == 0) count = 1;
  if (cudaMalloc(dst, sizeof(T) * count) != cudaSuccess) return sg_fail(h, SG_E_ALLOC, "device allocation failed");
  SG_CUDA(h, cudaMemcpy(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice));
  return SG_OK;
}

int upload_terms(sg_ctx* h, TermTable& T, int which) {
  std::vector<int> rp, tj, tk;
  std::vector<double> tg;
  build_terms(h, which, rp, tj, tk, tg);
  T.nnz = (int)tj.size();
  if (tj.empty()) { tj.push_back(0); tk.push_back(0); tg.push_back(0.0); }
  std::vector<float> tgf(tg.begin(), tg.end());
  std::vector<float> tgd;
  for (double v : tg) {
    const df2 d = df_from_double(v);
    tgd.push_back(d.hi), tgd.push_back(d.lo);
  }
  // weight slot of each term: 0 for the mean term, 1 + (k-1) p + n for c_k gamma(n), n = min(alpha_k, beta_k)
  std::vector<int> tw(tj.size(), 0);
  for (int i = 0; i + 1 < (int)rp.size(); ++i)
    for (int t = rp[i]; t < rp[i + 1]; ++t) {
      const int k = tk[t];
      if (k == 0) continue;
      const int ai = h->alpha[(size_t)i * h->M + k - 1], aj = h->alpha[(size_t)tj[t] * h->M + k - 1];
      tw[t] = 1 + (k - 1) * h->p + std::min(ai, aj);
    }
  int rc;
  if ((rc = upload(h, &T.row_ptr, rp.data(), rp.size()))) return rc;
  if ((rc = upload(h, &T.j, tj.data(), tj.size()))) return rc;
  if ((rc = upload(h, &T.k, tk.data(), tk.size()))) return rc;
  if ((rc = upload(h, &T.g, tg.data(), tg.size()))) return rc;
  if ((rc = upload(h, &T.gf, tgf.data(), tgf.size()))) return rc;
  if ((rc = upload(h, &T.gdf, tgd.data(), tgd.size()))) return rc;
  if ((rc = upload(h, &T.ws, tw.data(), tw.size()))) return rc;
  return SG_OK;
}

// Weight tables W[slot][e] = c_k(e) gamma(n) (slot 0: c_0) in double-float and in FP64, each when
// it fits in 2 GB: the operator then reads the product of a term instead of forming it.
int upload_weights(sg_ctx* h) {
  const size_t slots = 1 + (size_t)h->M * h->p;
  if (slots * h->Nc * 8 > (size_t)2 << 30) return SG_OK;
  {
    std::vector<double> w(slots * h->Nc);
    std::copy(h->coef_h.begin(), h->coef_h.begin() + h->Nc, w.begin());
    for (int k = 1; k <= h->M; ++k)
      for (int nn = 0; nn < h->p; ++nn) {
        const size_t s = 1 + (size_t)(k - 1) * h->p + nn;
        const double gm = gamma_1d(h->family, nn);
        for (size_t e = 0; e < h->Nc; ++e) w[s * h->Nc + e] = h->coef_h[(size_t)k * h->Nc + e] * gm;
      }
    const int rc = upload(h, &h->w64, w.data(), w.size());
    if (rc) return rc;
  }
  std::vector<float> w(2 * slots * h->Nc);
  for (size_t e = 0; e < h->Nc; ++e) {
    const df2 d = df_from_double(h->coef_h[e]);
    w[2 * e] = d.hi, w[2 * e + 1] = d.lo;
  }
  for (int k = 1; k <= h->M; ++k)
    for (int nn = 0; nn < h->p; ++nn) {
      const size_t s = 1 + (size_t)(k - 1) * h->p + nn;
      const double gm = gamma_1d(h->family, nn);
      for (size_t e = 0; e < h->Nc; ++e) {
        const df2 d = df_from_double(h->coef_h[(size_t)k * h->Nc + e] * gm);
        w[2 * (s * h->Nc + e)] = d.hi, w[2 * (s * h->Nc + e) + 1] = d.lo;
      }
    }
  return upload(h, &h->wdf, w.data(), w.size());
}

void free_terms(TermTable& T) {
  cudaFree(T.row_ptr), cudaFree(T.j), cudaFree(T.k), cudaFree(T.g), cudaFree(T.gf), cudaFree(T.gdf), cudaFree(T.ws);
  T = TermTable{};
}

// FP64 operator on all rows: Y = A X (R == nullptr) or Y = R - A X, R FP64
int apply_f64(sg_ctx* h, int which, int xprec, const void* X, int yprec, void* Y, const double* R) {
  return launch_apply(h, which, xprec, X, 0, yprec, Y, 0, SG_F64, R, 0, 0, h->P, 0, 0, SG_F64);
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// page-locked host memory (an asynchronous copy into pageable memory would block the host)
bool is_pinned_host(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

// early copy of the current iterate U (device, N doubles) to h->spec_dst, on the side stream
int spec_copy_u(sg_ctx* h, const double* U, size_t N) {
  if (!h->spec_dst) return SG_OK;
  if (!h->cstream) {
    SG_CUDA(h, cudaStreamCreateWithFlags(&h->cstream, cudaStreamNonBlocking));
    SG_CUDA(h, cudaEventCreateWithFlags(&h->ev_u, cudaEventDisableTiming));
    SG_CUDA(h, cudaEventCreateWithFlags(&h->ev_c, cudaEventDisableTiming));
  }
  SG_CUDA(h, cudaEventRecord(h->ev_u, h->stream));
  SG_CUDA(h, cudaStreamWaitEvent(h->cstream, h->ev_u, 0));
  SG_CUDA(h, cudaMemcpyAsync(h->spec_dst, U, sizeof(double) * N, cudaMemcpyDeviceToHost, h->cstream));
  SG_CUDA(h, cudaEventRecord(h->ev_c, h->cstream));
  h->spec_pending = true;
  return SG_OK;
}

// before U changes: make the main stream wait for an early copy still reading it
int spec_invalidate(sg_ctx* h) {
  if (!h->spec_pending) return SG_OK;
  SG_CUDA(h, cudaStreamWaitEvent(h->stream, h->ev_c, 0));
  h->spec_pending = false;
  return SG_OK;
}

double host_dot(sg_ctx* h, const double* x, const double* y, size_t N, int* rc) {
  const double* xs[1] = {x};
  const void* ys[1] = {y};
  int yp[1] = {SG_F64};
  double out = 0;
  *rc = vec_dot_pairs(h, 1, xs, ys, yp, N, &out);
  return out;
}

int precond_blocktri_exact(sg_ctx* h, const double* R, double* Z, int transpose);

int apply_precond(sg_ctx* h, int pc, int rprec, const void* R, void* Z, int prec, int transpose) {
  if (pc == SG_PC_BLOCKTRI_EXACT) {
    if (rprec != SG_F64 || prec != SG_F64) return sg_fail(h, SG_E_ARG, "exact block-triangular preconditioner: FP64 only");
    const int rc = precond_blocktri_exact(h, (const double*)R, (double*)Z, transpose);
    return rc == SG_E_NOCONV ? SG_OK : rc;       // an inner solve at its limit still gives a usable Z
  }
  if (pc == SG_PC_BLOCKTRI) return precond_blocktri(h, rprec, R, Z, prec, transpose);
  if (pc == SG_PC_BLOCKDIAG) return precond_blockdiag(h, rprec, R, Z, prec);
  if (pc == SG_PC_BLOCKSYM) return precond_blocksym(h, rprec, R, Z, prec);
  if (pc == SG_PC_BLOCKSYM_REC) return precond_blocksym_rec(h, rprec, R, Z, prec);
  return vec_cast(h, rprec, R, zprec_of(prec), Z, h->Nx * (size_t)h->P);
}

// Krylov vectors use the padded length Np (multiple of 64) with zero padding, so the
// Gram-Schmidt kernels can run 16-byte loads over whole vectors.
// Krylov workspace.  layout: 0 = FP64 basis, 1 = double-float basis, -1 = the basis is not
// used.  The Gram-Schmidt kernels stream whole padded vectors and rely on zero padding, which
// the other layout's vectors do not leave behind, so a change of layout clears the basis.
int ensure_krylov(sg_ctx* h, int nv, int nz, int zprec, int layout = -1) {
  const size_t Np = h->Np;
  if (h->kv_cap < nv) {
    cudaFree(h->kv);
    h->kv = nullptr;
    h->kv_cap = 0;
    if (cudaMalloc(&h->kv, sizeof(double) * Np * nv) != cudaSuccess) return sg_fail(h, SG_E_ALLOC, "alloc Krylov basis");
    SG_CUDA(h, cudaMemsetAsync(h->kv, 0, sizeof(double) * Np * nv, h->stream));
    h->kv_cap = nv;
    h->kv_layout = layout;
  }
  if (layout >= 0 && h->kv_layout != layout) {
    SG_CUDA(h, cudaMemsetAsync(h->kv, 0, sizeof(double) * Np * h->kv_cap, h->stream));
    h->kv_layout = layout;
  }
  if (h->kz_cap < nz || h->kz_prec != zprec) {
    cudaFree(h->kz);
    h->kz = nullptr;
    h->kz_cap = 0;
    // preconditioned vectors at the padded stride Np, so every z_j starts 128-byte aligned
    if (cudaMalloc(&h->kz, prec_size(zprec) * Np * std::max(nz, 1)) != cudaSuccess)
      return sg_fail(h, SG_E_ALLOC, "alloc preconditioned basis");
    h->kz_cap = std::max(nz, 1);
    h->kz_prec = zprec;
  }
  if (!h->qmax && cudaMalloc(&h->qmax, sizeof(unsigned) * (SG_MAX_RESTART + 1) * (size_t)h->P) != cudaSuccess)
    return sg_fail(h, SG_E_ALLOC, "alloc grid maxima");
  if (!h->ktmp) {
    if (cudaMalloc(&h->ktmp, sizeof(double) * Np * 4) != cudaSuccess) return sg_fail(h, SG_E_ALLOC, "alloc work vectors");
    SG_CUDA(h, cudaMemsetAsync(h->ktmp, 0, sizeof(double) * Np * 4, h->stream));
  }
  return ensure_reduction(h);
}

// ---------------------------------------------------------------------------
// Restarted right-preconditioned GMRES / FGMRES (Saad-Schultz; Sec. 4.2, 6).
// The Arnoldi / Givens / restart logic is shared; the vector storage and
// arithmetic come from an Ops class: OpsF64 (IEEE FP64 basis) or OpsDF (double-float
// basis, FGMRES only).  Ops::v(l) is basis vector l; reductions land in the
// reduction slots (0: Gram-Schmidt coefficients, 1: squared norm).
struct OpsF64 {
  sg_ctx* h;
  const sg_solve_opts& o;
  size_t N;
  const double* F;
  double* U;
  bool flexible;
  bool dfop;       // the outer operator A z_j in double-float arithmetic (FP32/BF16 z_j, FP64 result)
  double* V;
  int init() {
    int rc = ensure_krylov(h, o.restart + 1, flexible ? o.restart : 1, zprec_of(o.pc_prec), 0);
    V = h->kv;
    return rc;
  }
  double* v(int l) { return V + h->Np * l; }
  void* z(int j) { return (char*)h->kz + prec_size(zprec_of(o.pc_prec)) * h->Np * (flexible ? j : 0); }
  int norm2_rhs(double* out) { int rc; *out = host_dot(h, F, F, N, &rc); return rc; }
  int zero_solution() { return vec_fill(h, U, N, 0.0); }
  int residual(bool u_zero) {
    if (u_zero) {                                               // F - A 0 = F: no operator pass
      SG_CUDA(h, cudaMemcpyAsync(v(0), F, sizeof(double) * N, cudaMemcpyDeviceToDevice, h->stream));
      return SG_OK;
    }
    int rc;
    if ((rc = spec_copy_u(h, U, N))) return rc;                 // U is final if this check converges
    return apply_f64(h, 0, SG_F64, U, SG_F64, v(0), F);
  }
  int norm2(int l, double* out) { int rc; *out = host_dot(h, v(l), v(l), N, &rc); return rc; }
  // FP32 z_j are read through their blocks' fixed-point grids (SG_F32Q) by the operator and by the
  // solution update alike, so the flexible basis is the grid values z'_j (the flexible method takes
  // whatever z_j it is given); the double-float operator then forms cell features by exact FP32
  // differences instead of error-free sums.  The block maxima of z_j are kept for the update.
  bool quant() const { return dfop && flexible && zprec_of(o.pc_prec) == SG_F32; }
  unsigned* qm(int j) const { return h->qmax + (size_t)j * h->P; }
  int precond(int j) {
    h->zmax_out = quant() ? qm(j) : nullptr;
    h->zmax_done = false;
    int rc = apply_precond(h, o.precond, SG_F64, v(j), z(j), o.pc_prec, o.transpose);
    h->zmax_out = nullptr;
    if (rc || !quant() || h->zmax_done) return rc;
    return block_absmax(h, (const float*)z(j), qm(j));
  }
  int apply(int j) {
    if (dfop) {  // FP32-class z_j is exact in double-float; w is rounded once to FP64 on the store
      h->qcur = quant() ? qm(j) : nullptr;
      return launch_apply(h, 0, quant() ? SG_F32Q : zprec_of(o.pc_prec), z(j), 0, SG_F64, v(j + 1), 0, SG_F64,
                          nullptr, 0, 0, h->P, 0, 0, SG_DF64);
    }
    return apply_f64(h, 0, zprec_of(o.pc_prec), z(j), SG_F64, v(j + 1), nullptr);
  }
  int dots(int j, bool ww) { return vec_dots(h, V, h->Np, j + 1, v(j + 1), h->Np, ww, nullptr); }
  int axpys(int j, const double* c) { return vec_axpys_norm(h, V, h->Np, j + 1, c, v(j + 1), h->Np, nullptr); }
  int update(int k, const double* y) {
    int rc0 = spec_invalidate(h);
    if (rc0) return rc0;
    if (quant()) return vec_update_q(h, U, (const float*)h->kz, h->Np, k, y, N, h->qmax);
    if (flexible) return vec_update(h, U, zprec_of(o.pc_prec), h->kz, h->Np, k, y, N);
    double* t = h->ktmp;
    SG_CUDA(h, cudaMemsetAsync(t, 0, sizeof(double) * N, h->stream));
    int rc;
    if ((rc = vec_update(h, t, SG_F64, V, h->Np, k, y, N))) return rc;
    if ((rc = apply_precond(h, o.precond, SG_F64, t, h->kz, o.pc_prec, o.transpose))) return rc;
    return vec_axpy_prec(h, 1.0, zprec_of(o.pc_prec), h->kz, U, N);
  }
  int finish() { return SG_OK; }
};

struct OpsDF {
  sg_ctx* h;
  const sg_solve_opts& o;
  size_t N;
  const double* F;
  double* U;
  float* V;    // vector l: hi at V + 2 Np l, lo at + Np
  float* Fd;   // right-hand side and solution in double-float
  float* Ud;
  int init() {
    if (o.pc_prec != SG_F32 && o.pc_prec != SG_BF16 && o.pc_prec != SG_BF16Z)
      return sg_fail(h, SG_E_ARG, "double-float mode needs an FP32 or BF16 preconditioner");
    int rc = ensure_krylov(h, o.restart + 1, o.restart, zprec_of(o.pc_prec), 1);
    if (rc) return rc;
    const size_t Np = h->Np;
    V = (float*)h->kv;
    Fd = (float*)h->ktmp;
    Ud = (float*)(h->ktmp + Np);
    if ((rc = df_from_f64(h, F, Fd, N, Np))) return rc;
    if (o.x0_given) return df_from_f64(h, U, Ud, N, Np);
    SG_CUDA(h, cudaMemsetAsync(Ud, 0, sizeof(float) * 2 * Np, h->stream));
    return SG_OK;
  }
  float* v(int l) { return V + 2 * h->Np * l; }
  void* z(int j) { return (char*)h->kz + prec_size(zprec_of(o.pc_prec)) * h->Np * j; }
  int norm2_rhs(double* out) {
    int rc;
    if ((rc = df_dots(h, nullptr, 0, 0, Fd, h->Np, true))) return rc;
    return copy_red(h, 0, 1, out);
  }
  int zero_solution() { return vec_fill(h, U, N, 0.0); }
  int residual(bool u_zero) {
    const size_t Np = h->Np;
    if (u_zero) {
      SG_CUDA(h, cudaMemcpyAsync(v(0), Fd, sizeof(float) * 2 * Np, cudaMemcpyDeviceToDevice, h->stream));
      return SG_OK;
    }
    // restart (and final check): the true residual of the FP64 iterate in IEEE FP64, then split
    int rc;
    double* r64 = h->ktmp + 2 * Np;
    if ((rc = spec_invalidate(h))) return rc;
    if ((rc = df_to_f64(h, Ud, U, N, Np))) return rc;
    if ((rc = spec_copy_u(h, U, N))) return rc;                // U is final if this check converges
    if ((rc = apply_f64(h, 0, SG_F64, U, SG_F64, r64, F))) return rc;
    return df_from_f64(h, r64, v(0), N, Np);
  }
  int norm2(int l, double* out) {
    int rc;
    if ((rc = df_dots(h, nullptr, 0, 0, v(l), h->Np, true))) return rc;
    return copy_red(h, 0, 1, out);
  }
  bool quant() const { return zprec_of(o.pc_prec) == SG_F32; }     // grid-read z_j, as in OpsF64
  unsigned* qm(int j) const { return h->qmax + (size_t)j * h->P; }
  int precond(int j) {
    int rc = apply_precond(h, o.precond, SG_F32, v(j), z(j), o.pc_prec, o.transpose);
    if (rc || !quant()) return rc;
    return block_absmax(h, (const float*)z(j), qm(j));
  }
  int apply(int j) {
    h->qcur = quant() ? qm(j) : nullptr;
    return launch_apply(h, 0, quant() ? SG_F32Q : zprec_of(o.pc_prec), z(j), 0, SG_DF64, v(j + 1), h->Np, SG_DF64,
                        nullptr, 0, 0, h->P, 0, 0, SG_DF64);
  }
  int dots(int j, bool ww) { return df_dots(h, V, 2 * h->Np, j + 1, v(j + 1), h->Np, ww); }
  int axpys(int j, const double* c) { return df_axpys_norm(h, V, 2 * h->Np, j + 1, c, v(j + 1), h->Np); }
  int update(int k, const double* y) {
    if (quant()) return df_update_q(h, Ud, h->Np, (const float*)h->kz, h->Np, k, y, N, h->qmax);
    return df_update(h, Ud, h->Np, zprec_of(o.pc_prec), h->kz, h->Np, k, y, N);
  }
  int finish() {
    if (h->true_res_valid) return SG_OK;       // the converged check already wrote this iterate to U
    int rc = spec_invalidate(h);
    return rc ? rc : df_to_f64(h, Ud, U, N, h->Np);
  }
};

// The basis is normalised lazily: the stored vector l is v_l / s_l with s_l = 1 / ||stored
// v_l||, and every consumer folds s_l into its scalars (the preconditioner and the operator
// are linear, so z_j and A z_j carry the factor s_j), which saves one read-write pass over
// a basis vector per iteration.
template <class Ops>
int solve_gmres_t(sg_ctx* h, Ops& ops, const sg_solve_opts& o, sg_solve_info& info) {
  const int m = o.restart;
  int rc = ops.init();
  if (rc) return rc;
  double bb = 0;
  if ((rc = ops.norm2_rhs(&bb))) return rc;
  const double bnorm = std::sqrt(bb);
  if (!std::isfinite(bnorm)) return sg_fail(h, SG_E_NONFINITE, "non-finite right-hand side");
  if (bnorm == 0.0) {
    info.relres_true = info.relres_est = 0;
    return ops.zero_solution();
  }
  std::vector<double> H((m + 1) * m), cs(m), sn(m), g(m + 1), dv(m + 2), d2(m + 2), coef(m + 1), y(m), sc(m + 1);
  int its = 0;
  bool u_zero = !o.x0_given;
  for (;;) {
    {
      PhaseScope ps(h, 3);
      if ((rc = ops.residual(u_zero))) return rc;   // stored v_0 = F - A U, the IEEE FP64 true residual
    }
    double b2 = 0;
    if ((rc = ops.norm2(0, &b2))) return rc;
    const double beta = std::sqrt(b2);
    if (!std::isfinite(beta)) return sg_fail(h, SG_E_NONFINITE, "non-finite residual");
    info.relres_true = beta / bnorm;
    if (beta <= o.tol * bnorm) {
      info.relres_est = info.relres_true;
      h->true_res_valid = true;    // the caller need not recompute it
      break;
    }
    if (its >= o.maxit) { info.iters = its; ops.finish(); return SG_E_NOCONV; }
    sc[0] = 1.0 / beta;
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int k = 0;
    for (int j = 0; j < m; ++j) {
      {
        PhaseScope ps(h, 1);
        if ((rc = ops.precond(j))) return rc;                  // z_j / s_j = B^{-1} (stored v_j)
      }
      {
        PhaseScope ps(h, 0);
        if ((rc = ops.apply(j))) return rc;                    // w / s_j = A z_j / s_j, stored in v_{j+1}
      }
      // classical Gram-Schmidt on the stored vectors: d = V^T w (and w.w), w -= V (s^2 d), ||w||^2
      {
        PhaseScope ps(h, 2);
        if ((rc = ops.dots(j, true))) return rc;
      }
      if ((rc = copy_red(h, 0, j + 2, dv.data()))) return rc;
      for (int i = 0; i <= j; ++i) coef[i] = sc[i] * sc[i] * dv[i];
      if ((rc = upload_red(h, 3, coef.data(), j + 1))) return rc;
      double nrm2 = 0;
      {
        PhaseScope ps(h, 2);
        if ((rc = ops.axpys(j, red_slot(h, 3)))) return rc;
      }
      if ((rc = copy_red(h, 1, 1, &nrm2))) return rc;
      if (o.reorth && nrm2 < 0.5 * dv[j + 1]) {
        {
          PhaseScope ps(h, 2);
          if ((rc = ops.dots(j, false))) return rc;
        }
        if ((rc = copy_red(h, 0, j + 1, d2.data()))) return rc;
        for (int i = 0; i <= j; ++i) coef[i] = sc[i] * sc[i] * d2[i];
        if ((rc = upload_red(h, 3, coef.data(), j + 1))) return rc;
        {
          PhaseScope ps(h, 2);
          if ((rc = ops.axpys(j, red_slot(h, 3)))) return rc;
        }
        if ((rc = copy_red(h, 1, 1, &nrm2))) return rc;
        for (int i = 0; i <= j; ++i) dv[i] += d2[i];
      }
      const double hn = sc[j] * std::sqrt(nrm2);
      for (int i = 0; i <= j; ++i) {
        const double hij = sc[i] * sc[j] * dv[i];
        if (!std::isfinite(hij)) return sg_fail(h, SG_E_NONFINITE, "non-finite Hessenberg entry");
        H[i * m + j] = hij;
      }
      if (!std::isfinite(hn)) return sg_fail(h, SG_E_NONFINITE, "non-finite Arnoldi norm");
      H[(j + 1) * m + j] = hn;
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
        H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
        H[i * m + j] = t;
      }
      const double d = std::hypot(H[j * m + j], H[(j + 1) * m + j]);
      if (d == 0.0) return sg_fail(h, SG_E_BREAKDOWN, "GMRES breakdown (zero Hessenberg column)");
      cs[j] = H[j * m + j] / d;
      sn[j] = H[(j + 1) * m + j] / d;
      H[j * m + j] = d;
      H[(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++its;
      k = j + 1;
      info.relres_est = std::fabs(g[j + 1]) / bnorm;
      if (hn == 0.0 || std::fabs(g[j + 1]) <= o.tol * bnorm || its >= o.maxit) break;
      sc[j + 1] = 1.0 / std::sqrt(nrm2);
    }
    for (int i = k - 1; i >= 0; --i) {   // back substitution H y = g
      double s = g[i];
      for (int l = i + 1; l < k; ++l) s -= H[i * m + l] * y[l];
      y[i] = s / H[i * m + i];
    }
    for (int i = 0; i < k; ++i) y[i] *= sc[i];    // stored z_i = z_i / s_i
    {
      PhaseScope ps(h, 3);
      if ((rc = ops.update(k, y.data()))) return rc;
    }
    u_zero = false;
    info.restarts++;
  }
  info.iters = its;
  return ops.finish();
}

int solve_gmres(sg_ctx* h, const double* F, double* U, const sg_solve_opts& o, sg_solve_info& info, bool flexible) {
  const size_t N = h->Nx * (size_t)h->P;
  if (o.arith == SG_ARITH_DF64) {
    if (!flexible) return sg_fail(h, SG_E_ARG, "double-float mode is implemented for FGMRES");
    OpsDF ops{h, o, N, F, U, nullptr, nullptr, nullptr};
    return solve_gmres_t(h, ops, o, info);
  }
  OpsF64 ops{h, o, N, F, U, flexible, o.arith == SG_ARITH_F64_DFOP, nullptr};
  return solve_gmres_t(h, ops, o, info);
}

// ---------------------------------------------------------------------------
// GPCG[1] (Sec. 4.2, 6): g = B^{-1} r, A-orthogonalise against the previous
// direction, alpha = <r,d>/<Ad,d>.
int solve_gpcg(sg_ctx* h, const double* F, double* U, const sg_solve_opts& o, sg_solve_info& info) {
  const size_t N = h->Nx * (size_t)h->P;
  const int pcm = o.pc_prec, zp = zprec_of(pcm);     // preconditioner mode, storage of z
  int rc = ensure_krylov(h, 1, 1, zp);
  if (rc) return rc;
  double *r = h->ktmp, *Ag = h->ktmp + N, *d = h->ktmp + 2 * N, *Ad = h->ktmp + 3 * N;
  void* gv = h->kz;
  const double bnorm = std::sqrt(host_dot(h, F, F, N, &rc));
  if (rc) return rc;
  if (bnorm == 0.0) return vec_fill(h, U, N, 0.0);
  if ((rc = apply_f64(h,0, SG_F64, U, SG_F64, r, F))) return rc;
  double rr = host_dot(h, r, r, N, &rc);
  if (rc) return rc;
  double Add_prev = 0;
  int its = 0;
  while (std::sqrt(rr) > o.tol * bnorm) {
    if (!std::isfinite(rr)) return sg_fail(h, SG_E_NONFINITE, "non-finite residual");
    if (its >= o.maxit) { info.iters = its; info.relres_true = std::sqrt(rr) / bnorm; return SG_E_NOCONV; }
    if ((rc = apply_precond(h, o.precond, SG_F64, r, gv, pcm, o.transpose))) return rc;
    if ((rc = apply_f64(h,0, zp, gv, SG_F64, Ag, nullptr))) return rc;
    if (its == 0) {
      if ((rc = vec_cast(h, zp, gv, SG_F64, d, N))) return rc;
      SG_CUDA(h, cudaMemcpyAsync(Ad, Ag, sizeof(double) * N, cudaMemcpyDeviceToDevice, h->stream));
    } else {
      const double beta = host_dot(h, Ag, d, N, &rc) / Add_prev;
      if (rc) return rc;
      if ((rc = vec_axpby(h, 0.0, d, -beta, d, N))) return rc;        // d = -beta d
      if ((rc = vec_axpy_prec(h, 1.0, zp, gv, d, N))) return rc;      // d += g
      if ((rc = vec_axpby(h, 1.0, Ag, -beta, Ad, N))) return rc;      // Ad = Ag - beta Ad
    }
    const double* xs[2] = {r, Ad};
    const void* ys[2] = {d, d};
    int yp[2] = {SG_F64, SG_F64};
    double dd[2];
    if ((rc = vec_dot_pairs(h, 2, xs, ys, yp, N, dd))) return rc;
    if (!(dd[1] > 0) && !(dd[1] < 0)) return sg_fail(h, SG_E_BREAKDOWN, "GPCG breakdown (<Ad,d> = 0)");
    const double alpha = dd[0] / dd[1];
    Add_prev = dd[1];
    if ((rc = vec_axpby(h, alpha, d, 1.0, U, N))) return rc;
    if ((rc = vec_axpby(h, -alpha, Ad, 1.0, r, N))) return rc;
    rr = host_dot(h, r, r, N, &rc);
    if (rc) return rc;
    ++its;
  }
  info.iters = its;
  info.relres_est = std::sqrt(rr) / bnorm;
  return SG_OK;
}

// Standard PCG (Sec. 4.2, with B_D or the SPD B_S); B_T is accepted but not SPD.
// Stationary block Gauss-Seidel (Sec. 4.2, the B-GS rows of Table 3): U += B^{-1}(F - A U).
int solve_bgs(sg_ctx* h, const double* F, double* U, const sg_solve_opts& o, sg_solve_info& info) {
  const size_t N = h->Nx * (size_t)h->P;
  const int pcm = o.pc_prec, zp = zprec_of(pcm);     // preconditioner mode, storage of z
  int rc = ensure_krylov(h, 1, 1, zp);
  if (rc) return rc;
  double* r = h->ktmp;
  const double bnorm = std::sqrt(host_dot(h, F, F, N, &rc));
  if (rc) return rc;
  if (!std::isfinite(bnorm)) return sg_fail(h, SG_E_NONFINITE, "non-finite right-hand side");
  if (bnorm == 0.0) return vec_fill(h, U, N, 0.0);
  int its = 0;
  for (;;) {
    if ((rc = apply_f64(h, 0, SG_F64, U, SG_F64, r, F))) return rc;
    const double rr = host_dot(h, r, r, N, &rc);
    if (rc) return rc;
    if (!std::isfinite(rr)) return sg_fail(h, SG_E_NONFINITE, "non-finite residual");
    info.relres_true = info.relres_est = std::sqrt(rr) / bnorm;
    if (std::sqrt(rr) <= o.tol * bnorm) { h->true_res_valid = true; break; }
    if (its >= o.maxit) { info.iters = its; return SG_E_NOCONV; }
    {
      PhaseScope ps(h, 1);
      if ((rc = apply_precond(h, o.precond, SG_F64, r, h->kz, pcm, o.transpose))) return rc;
    }
    if ((rc = vec_axpy_prec(h, 1.0, zp, h->kz, U, N))) return rc;
    ++its;
  }
  info.iters = its;
  return SG_OK;
}

int solve_pcg(sg_ctx* h, const double* F, double* U, const sg_solve_opts& o, sg_solve_info& info) {
  const size_t N = h->Nx * (size_t)h->P;
  const int pcm = o.pc_prec, zp = zprec_of(pcm);     // preconditioner mode, storage of z
  int rc = ensure_krylov(h, 1, 1, zp);
  if (rc) return rc;
  double *r = h->ktmp, *Ad = h->ktmp + N, *d = h->ktmp + 2 * N;
  void* z = h->kz;
  const double bnorm = std::sqrt(host_dot(h, F, F, N, &rc));
  if (rc) return rc;
  if (bnorm == 0.0) return vec_fill(h, U, N, 0.0);
  if ((rc = apply_f64(h,0, SG_F64, U, SG_F64, r, F))) return rc;
  if ((rc = apply_precond(h, o.precond, SG_F64, r, z, pcm, o.transpose))) return rc;
  if ((rc = vec_cast(h, zp, z, SG_F64, d, N))) return rc;
  const double* xs0[2] = {r, r};
  const void* ys0[2] = {z, r};
  int yp0[2] = {zp, SG_F64};
  double t2[2];
  if ((rc = vec_dot_pairs(h, 2, xs0, ys0, yp0, N, t2))) return rc;
  double rz = t2[0], rr = t2[1];
  int its = 0;
  while (std::sqrt(rr) > o.tol * bnorm) {
    if (!std::isfinite(rr)) return sg_fail(h, SG_E_NONFINITE, "non-finite residual");
    if (its >= o.maxit) { info.iters = its; info.relres_true = std::sqrt(rr) / bnorm; return SG_E_NOCONV; }
    if ((rc = apply_f64(h,0, SG_F64, d, SG_F64, Ad, nullptr))) return rc;
    const double dAd = host_dot(h, d, Ad, N, &rc);
    if (rc) return rc;
    if (!(dAd > 0) && !(dAd < 0)) return sg_fail(h, SG_E_BREAKDOWN, "PCG breakdown (<d,Ad> = 0)");
    const double alpha = rz / dAd;
    if ((rc = vec_axpby(h, alpha, d, 1.0, U, N))) return rc;
    if ((rc = vec_axpby(h, -alpha, Ad, 1.0, r, N))) return rc;
    ++its;
    if ((rc = apply_precond(h, o.precond, SG_F64, r, z, pcm, o.transpose))) return rc;
    if ((rc = vec_dot_pairs(h, 2, xs0, ys0, yp0, N, t2))) return rc;
    const double beta = t2[0] / rz;
    rz = t2[0], rr = t2[1];
    if ((rc = vec_axpby(h, 0.0, d, beta, d, N))) return rc;           // d = beta d
    if ((rc = vec_axpy_prec(h, 1.0, zp, z, d, N))) return rc;          // d += z
  }
  info.iters = its;
  info.relres_est = std::sqrt(rr) / bnorm;
  return SG_OK;
}

// The 2 x 2 block-triangular preconditioner with the exact lower-degree block (Sec. 4.2, Theorem 1).
// The PC basis is degree-graded, so the first lvl_off[p] blocks of an SG vector are a vector of the
// degree-(p-1) system A_hat = A_{p-1}, solved on a child handle of that degree.
int precond_blocktri_exact(sg_ctx* h, const double* R, double* Z, int transpose) {
  int rc;
  if (h->p == 0) return precond_blocktri(h, SG_F64, R, Z, SG_F64, transpose);
  if (!h->child) {
    sg_problem pr{h->n, h->M, h->p - 1, h->family, h->coef_h.data(), h->nu1, h->nu2, h->omega, h->elements,
                  h->gs_order};
    sg_handle c = nullptr;
    if ((rc = sg_setup(&pr, h->stream, &c))) return sg_fail(h, rc, "exact block-triangular: set-up of the degree p-1 "
                                                                     "system failed: " + std::string(sg_last_error(nullptr)));
    h->child = c;
  }
  sg_ctx* c = h->child;
  c->stream = h->stream;
  if ((rc = ensure_prec_work(h, SG_F64))) return rc;
  const int nlow = h->lvl_off[h->p], np = h->P - nlow;
  const size_t Nx = h->Nx;
  sg_solve_opts io{};
  io.method = SG_FGMRES, io.precond = SG_PC_BLOCKTRI, io.restart = h->inner_restart, io.maxit = 2000;
  io.tol = h->inner_tol, io.pc_prec = SG_F64, io.transpose = transpose, io.arith = SG_ARITH_F64;
  sg_solve_info info{};
  const long long before = c->tr.launches[0] + c->tr.launches[1] + c->tr.launches[2] + c->tr.launches[3];
  int rin;
  if (!transpose) {
    rin = sg_solve(c, R, Z, &io, &info);                                          // Z_low = A_hat^{-1} R_low
    if (rin != SG_OK && rin != SG_E_NOCONV) return sg_fail(h, rin, std::string("exact block-triangular: ") + c->err);
    double* T = (double*)h->work[SG_F64].T;                                       // T = R_p - W Z_low
    if ((rc = launch_apply(h, 1, SG_F64, Z, 0, SG_F64, T, 0, SG_F64, R, 0, nlow, np, nlow, 0, SG_F64))) return rc;
    if ((rc = vcycle_run(h, SG_F64, np, T, SG_F64, Z + (size_t)nlow * Nx, true))) return rc;
  } else {
    if ((rc = vcycle_run(h, SG_F64, np, R + (size_t)nlow * Nx, SG_F64, Z + (size_t)nlow * Nx, false))) return rc;
    if (!h->xbuf && cudaMalloc(&h->xbuf, sizeof(double) * Nx * h->P) != cudaSuccess)
      return sg_fail(h, SG_E_ALLOC, "alloc exact block-triangular buffer");
    // T_low = R_low - W^T Z_p: only the degree p-1 rows couple to degree p
    const int r1 = h->lvl_off[h->p - 1], n1 = nlow - r1;
    SG_CUDA(h, cudaMemcpyAsync(h->xbuf, R, sizeof(double) * Nx * r1, cudaMemcpyDeviceToDevice, h->stream));
    if ((rc = launch_apply(h, 2, SG_F64, Z, 0, SG_F64, h->xbuf + (size_t)r1 * Nx, 0, SG_F64, R, 0, r1, n1, r1, 0,
                           SG_F64)))
      return rc;
    rin = sg_solve(c, h->xbuf, Z, &io, &info);                                    // Z_low = A_hat^{-T} T_low
    if (rin != SG_OK && rin != SG_E_NOCONV) return sg_fail(h, rin, std::string("exact block-triangular: ") + c->err);
  }
  const long long after = c->tr.launches[0] + c->tr.launches[1] + c->tr.launches[2] + c->tr.launches[3];
  count_launch(h, (int)(after - before));
  return rin;
}

void destroy_ctx(sg_ctx* h) {
  if (!h) return;
  if (h->child) {
    destroy_ctx(h->child);
    h->child = nullptr;
  }
  cudaFree(h->xbuf);
  cudaFree(h->ew), cudaFree(h->p1w), cudaFree(h->bsr);
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second.exec);
  h->graphs.clear();
  cudaFree(h->coef64), cudaFree(h->coef32), cudaFree(h->coefdf), cudaFree(h->wdf), cudaFree(h->w64), cudaFree(h->pvec);
  cudaFree(h->qmax);
  free_terms(h->t_all), free_terms(h->t_lower), free_terms(h->t_upper), free_terms(h->t_off), free_terms(h->t_diag);
  for (int l = 0; l < SG_MAX_LEVELS; ++l) cudaFree(h->lev[l].st64), cudaFree(h->lev[l].st32);
  for (auto& W : h->work) {
    sg_gfree(W.T), sg_gfree(W.T32), cudaFree(W.S1), cudaFree(W.S2);
    for (int l = 0; l < SG_MAX_LEVELS; ++l) sg_gfree(W.b[l]), sg_gfree(W.x[l]);
  }
  cudaFree(h->red_partial), cudaFree(h->red_out), cudaFree(h->red_count), cudaFreeHost(h->red_host);
  cudaFree(h->kv), cudaFree(h->kz), cudaFree(h->ktmp), cudaFree(h->dstage);
  if (h->cstream) cudaStreamDestroy(h->cstream);
  if (h->ev_u) cudaEventDestroy(h->ev_u);
  if (h->ev_c) cudaEventDestroy(h->ev_c);
  delete h;
}
}  // namespace

int apply_precond_ext(sg_ctx* h, int pc, int rprec, const void* R, void* Z, int prec, int transpose) {
  return apply_precond(h, pc, rprec, R, Z, prec, transpose);
}
int ensure_krylov_ext(sg_ctx* h, int nv, int nz, int zprec, int layout) { return ensure_krylov(h, nv, nz, zprec, layout); }

int sg_fail(sg_ctx* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  else {
    std::lock_guard<std::mutex> lk(g_err_mu);
    g_setup_err = msg;
  }
  return code;
}

int sg_check_device(sg_ctx* h, const char* who) {
  int dev = -1;
  const cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return sg_fail(h, SG_E_CUDA, std::string(who) + ": cudaGetDevice: " + cudaGetErrorString(e));
  if (dev != h->device)
    return sg_fail(h, SG_E_STATE, std::string(who) + ": the handle belongs to device " + std::to_string(h->device) +
                                      " but device " + std::to_string(dev) + " is current");
  return SG_OK;
}

size_t prec_size(int prec) {
  return (prec == SG_F64 || prec == SG_DF64) ? 8 : ((prec == SG_F32 || prec == SG_F32Q) ? 4 : 2);
}

extern "C" {

int sg_kl_coef(int n, int M, double sigma, double corr_len, const double* abar, double* coef_out, double* lambda_out) {
  if (n < 3 || M < 0 || M > 64 || !coef_out || !(corr_len > 0) || !std::isfinite(sigma))
    return sg_fail(nullptr, SG_E_ARG, "sg_kl_coef: bad argument");
  return kl_coef_host(n, M, sigma, corr_len, abar, coef_out, lambda_out);
}

int sg_kl_coef_p1(int n, int M, double sigma, double corr_len, double* coef_out, double* lambda_out) {
  if (n < 3 || M < 0 || M > 64 || !coef_out || !(corr_len > 0) || !std::isfinite(sigma))
    return sg_fail(nullptr, SG_E_ARG, "sg_kl_coef_p1: bad argument");
  return kl_coef_p1_host(n, M, sigma, corr_len, coef_out, lambda_out);
}

int sg_min_coef(int n, int M, const double* coef, double xi_max, double* amin_out) {
  if (n < 3 || M < 0 || !coef || !amin_out || !(xi_max >= 0) || !std::isfinite(xi_max))
    return sg_fail(nullptr, SG_E_ARG, "sg_min_coef: bad argument");
  const size_t Nc = (size_t)(n - 1) * (n - 1);
  double amin = INFINITY;
  for (size_t e = 0; e < Nc; ++e) {
    double s = 0;
    for (int k = 1; k <= M; ++k) s += std::fabs(coef[(size_t)k * Nc + e]);
    amin = std::min(amin, coef[e] - xi_max * s);
  }
  *amin_out = amin;
  return SG_OK;
}

int sg_rhs(sg_handle h, const double* f_nodes, double* F) {
  if (!h || !F) return h ? sg_fail(h, SG_E_ARG, "sg_rhs: null argument") : SG_E_ARG;
  if (const int rcd = sg_check_device(h, "sg_rhs")) return rcd;
  const double hh = 1.0 / (double)(h->n - 1);
  return vec_load(h, f_nodes, hh * hh, F);
}

const char* sg_last_error(sg_handle h) {
  if (h) return h->err.c_str();
  std::lock_guard<std::mutex> lk(g_err_mu);
  return g_setup_err.c_str();
}

int sg_setup(const sg_problem* prob, void* stream, sg_handle* out) {
  if (!prob || !out || !prob->coef) return sg_fail(nullptr, SG_E_ARG, "sg_setup: null argument");
  *out = nullptr;
  const int n = prob->n, M = prob->M, p = prob->p;
  bool pow2 = n >= 3 && n <= 4097 && ((n - 1) & (n - 2)) == 0;
  if (!pow2) return sg_fail(nullptr, SG_E_ARG, "sg_setup: n must be 2^L + 1 with 3 <= n <= 4097");
  if (M < 0 || M > 16 || p < 0 || p > 10) return sg_fail(nullptr, SG_E_ARG, "sg_setup: need 0 <= M <= 16, 0 <= p <= 10");
  if (prob->family != SG_LEGENDRE && prob->family != SG_HERMITE) return sg_fail(nullptr, SG_E_ARG, "sg_setup: bad family");
  const int nu1 = prob->nu1 ? prob->nu1 : 1, nu2 = prob->nu2 ? prob->nu2 : 1;
  if (nu1 < 1 || nu1 > 4 || nu2 < 1 || nu2 > 4) return sg_fail(nullptr, SG_E_ARG, "sg_setup: smoothing steps must be 1..4");
  double Pd = 1;
  for (int t = 1; t <= p; ++t) Pd = Pd * (M + t) / t;
  if (Pd > 4096) return sg_fail(nullptr, SG_E_ARG, "sg_setup: P exceeds 4096");
  sg_ctx* h = new sg_ctx();
  h->n = n, h->m = n - 2, h->M = M, h->p = p, h->family = prob->family;
  h->Nx = (size_t)h->m * h->m, h->Nc = (size_t)(n - 1) * (n - 1);
  h->nu1 = nu1, h->nu2 = nu2;
  h->omega = prob->omega > 0 ? prob->omega : 8.0 / 9.0;
  if (prob->elements != SG_Q1 && prob->elements != SG_P1) {
    delete h;
    return sg_fail(nullptr, SG_E_ARG, "sg_setup: elements must be SG_Q1 or SG_P1");
  }
  h->elements = prob->elements;
  if (prob->gs_order != SG_GS_LEX && prob->gs_order != SG_GS_RB) {
    delete h;
    return sg_fail(nullptr, SG_E_ARG, "sg_setup: gs_order must be SG_GS_LEX or SG_GS_RB");
  }
  h->gs_order = prob->gs_order;
  h->stream = (cudaStream_t)stream;
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return sg_fail(nullptr, SG_E_CUDA, "sg_setup: no current CUDA device");
  }
  build_basis(M, p, h->alpha, h->lvl_off);
  h->P = h->lvl_off.back();
  h->Np = (h->Nx * (size_t)h->P + 63) / 64 * 64;
  const size_t ncoef = (h->elements == SG_P1 ? 2 : 1) * h->Nc;     // per cell, or per triangle (SG_P1)
  h->coef_h.assign(prob->coef, prob->coef + (size_t)(M + 1) * ncoef);
  for (double v : h->coef_h)
    if (!std::isfinite(v)) { delete h; return sg_fail(nullptr, SG_E_ARG, "sg_setup: non-finite coefficient"); }
  h->const_mean = true;
  for (size_t e = 0; e < ncoef; ++e)
    if (h->coef_h[e] != 1.0) { h->const_mean = false; break; }
  int rc;
  std::vector<float> c32(h->coef_h.begin(), h->coef_h.end());
  std::vector<float> cdf;
  cdf.reserve(2 * h->coef_h.size());
  for (double v : h->coef_h) {
    const df2 d = df_from_double(v);
    cdf.push_back(d.hi), cdf.push_back(d.lo);
  }
  const bool q1 = h->elements == SG_Q1;
  if ((rc = upload(h, &h->coef64, h->coef_h.data(), h->coef_h.size())) ||
      (q1 && (rc = upload(h, &h->coef32, c32.data(), c32.size()))) ||
      (q1 && (rc = upload(h, &h->coefdf, cdf.data(), cdf.size()))) ||
      (rc = upload_terms(h, h->t_all, 0)) ||
      (rc = upload_terms(h, h->t_lower, 1)) || (rc = upload_terms(h, h->t_upper, 2)) ||
      (rc = upload_terms(h, h->t_off, 3)) || (rc = upload_terms(h, h->t_diag, 4)) || (q1 && (rc = upload_weights(h)))) {
    std::string e = h->err;
    destroy_ctx(h);
    return sg_fail(nullptr, rc, "sg_setup: " + e);
  }
  if (cudaMalloc(&h->pvec, sizeof(double) * std::max(h->P, 64)) != cudaSuccess) {
    destroy_ctx(h);
    return sg_fail(nullptr, SG_E_ALLOC, "sg_setup: scratch allocation");
  }
  // multigrid hierarchy n_{l+1} = (n_l + 1) / 2 down to n = 3
  h->nlev = 0;
  for (int nl = n;; nl = (nl + 1) / 2) {
    MGLevel& L = h->lev[h->nlev++];
    L.n = nl, L.m = nl - 2, L.N = (size_t)L.m * L.m;
    if (nl <= 3) break;
  }
  h->lc = 0;
  while (h->lc < h->nlev && h->lev[h->lc].n > 33) ++h->lc;
  if (h->elements == SG_P1) {
    if ((rc = setup_p1(h))) {
      std::string e = h->err;
      destroy_ctx(h);
      return sg_fail(nullptr, rc, "sg_setup: " + e);
    }
    *out = h;
    return SG_OK;
  }
  if (!h->const_mean) {
    std::vector<std::vector<double>> st;
    galerkin_stencils(n, h->nlev, h->coef_h.data(), st);
    for (int l = 0; l < h->nlev; ++l) {
      std::vector<float> s32(st[l].begin(), st[l].end());
      if ((rc = upload(h, &h->lev[l].st64, st[l].data(), st[l].size())) ||
          (rc = upload(h, &h->lev[l].st32, s32.data(), s32.size()))) {
        std::string e = h->err;
        destroy_ctx(h);
        return sg_fail(nullptr, rc, "sg_setup: " + e);
      }
    }
  }
  *out = h;
  return SG_OK;
}

void sg_destroy(sg_handle h) {
  if (h && h->stream) cudaStreamSynchronize(h->stream);
  destroy_ctx(h);
}

int sg_set_stream(sg_handle h, void* stream) {
  if (!h) return SG_E_ARG;
  h->stream = (cudaStream_t)stream;
  return SG_OK;
}

int sg_sizes(sg_handle h, int* Nx, int* P, int* nlevels) {
  if (!h) return SG_E_ARG;
  if (Nx) *Nx = (int)h->Nx;
  if (P) *P = h->P;
  if (nlevels) *nlevels = h->nlev;
  return SG_OK;
}

int sg_basis(sg_handle h, int* alpha) {
  if (!h || !alpha) return SG_E_ARG;
  std::copy(h->alpha.begin(), h->alpha.end(), alpha);
  return SG_OK;
}

int sg_apply(sg_handle h, const void* X, void* Y, int prec) {
  if (!h || !X || !Y || prec < 0 || prec > 3) return h ? sg_fail(h, SG_E_ARG, "sg_apply: bad argument") : SG_E_ARG;
  if (const int rcd = sg_check_device(h, "sg_apply")) return rcd;
  const size_t lo = prec == SG_DF64 ? h->Nx * (size_t)h->P : 0;
  const int arith = (prec == SG_F64 || prec == SG_DF64) ? prec : SG_F32;
  return launch_apply(h, 0, prec, X, lo, prec, Y, lo, SG_F64, nullptr, 0, 0, h->P, 0, 0, arith);
}

int sg_residual(sg_handle h, const double* F, const double* U, double* R) {
  if (!h || !F || !U || !R) return h ? sg_fail(h, SG_E_ARG, "sg_residual: null argument") : SG_E_ARG;
  if (const int rcd = sg_check_device(h, "sg_residual")) return rcd;
  if ((const void*)U == (const void*)R) return sg_fail(h, SG_E_ARG, "sg_residual: U must not alias R");
  return apply_f64(h,0, SG_F64, U, SG_F64, R, F);
}

int sg_precond_blocktri(sg_handle h, const double* R, void* Z, int prec, int transpose) {
  if (!h || !R || !Z || prec < 0 || prec > 4 || prec == SG_DF64) return h ? sg_fail(h, SG_E_ARG, "sg_precond_blocktri: bad argument") : SG_E_ARG;
  if (const int rcd = sg_check_device(h, "sg_precond_blocktri")) return rcd;
  return precond_blocktri(h, SG_F64, R, Z, prec, transpose != 0);
}

int sg_precond_blockdiag(sg_handle h, const double* R, void* Z, int prec) {
  if (!h || !R || !Z || prec < 0 || prec > 4 || prec == SG_DF64) return h ? sg_fail(h, SG_E_ARG, "sg_precond_blockdiag: bad argument") : SG_E_ARG;
  if (const int rcd = sg_check_device(h, "sg_precond_blockdiag")) return rcd;
  return precond_blockdiag(h, SG_F64, R, Z, prec);
}

int sg_precond_blocktri_exact(sg_handle h, const double* R, double* Z, int transpose, double inner_tol) {
  if (!h || !R || !Z || (const void*)R == (const void*)Z || !(inner_tol >= 0))
    return h ? sg_fail(h, SG_E_ARG, "sg_precond_blocktri_exact: bad argument") : SG_E_ARG;
  if (const int rcd = sg_check_device(h, "sg_precond_blocktri_exact")) return rcd;
  h->inner_tol = inner_tol > 0 ? inner_tol : 1e-12;
  h->inner_restart = 30;
  return precond_blocktri_exact(h, R, Z, transpose != 0);
}

int sg_precond_blocksym(sg_handle h, const double* R, void* Z, int prec) {
  if (!h || !R || !Z || prec < 0 || prec > 4 || prec == SG_DF64) return h ? sg_fail(h, SG_E_ARG, "sg_precond_blocksym: bad argument") : SG_E_ARG;
  if (const int rcd = sg_check_device(h, "sg_precond_blocksym")) return rcd;
  return precond_blocksym(h, SG_F64, R, Z, prec);
}

int sg_precond_blocksym_rec(sg_handle h, const double* R, double* Z) {
  if (!h || !R || !Z) return h ? sg_fail(h, SG_E_ARG, "sg_precond_blocksym_rec: null argument") : SG_E_ARG;
  if (const int rcd = sg_check_device(h, "sg_precond_blocksym_rec")) return rcd;
  return precond_blocksym_rec(h, SG_F64, R, Z, SG_F64);
}

int sg_vcycle(sg_handle h, const double* B, void* X, int nblocks, int prec) {
  if (!h || !B || !X || prec < 0 || prec > 4 || prec == SG_DF64 || nblocks < 0 || nblocks > h->P)
    return h ? sg_fail(h, SG_E_ARG, "sg_vcycle: bad argument") : SG_E_ARG;
  if (const int rcd = sg_check_device(h, "sg_vcycle")) return rcd;
  return vcycle_run(h, prec, nblocks, B, SG_F64, X);
}

static int solve_checked(sg_handle h, const double* F, double* U, const sg_solve_opts* opts, sg_solve_info* info_out);

// Every return of sg_solve leaves info (when given) describing the call: an error that stops the call
// before the solver has finished leaves it zeroed apart from its status.
int sg_solve(sg_handle h, const double* F, double* U, const sg_solve_opts* opts, sg_solve_info* info_out) {
  const int rc = solve_checked(h, F, U, opts, info_out);
  if (info_out) info_out->status = rc;
  return rc;
}

static int solve_checked(sg_handle h, const double* F, double* U, const sg_solve_opts* opts, sg_solve_info* info_out) {
  if (info_out) *info_out = sg_solve_info{};
  if (!h || !F || !U || !opts) return h ? sg_fail(h, SG_E_ARG, "sg_solve: null argument") : SG_E_ARG;
  if (const int rcd = sg_check_device(h, "sg_solve")) return rcd;
  sg_solve_opts o = *opts;
  if (o.method < SG_GMRES || o.method > SG_BGS || o.precond < 0 || o.precond > 5 || o.pc_prec < 0 || o.pc_prec > 4 ||
      o.pc_prec == SG_DF64 ||
      !(o.tol > 0) || o.maxit < 0)
    return sg_fail(h, SG_E_ARG, "sg_solve: bad options");
  if ((o.method == SG_GMRES || o.method == SG_FGMRES) && (o.restart < 1 || o.restart > 32))
    return sg_fail(h, SG_E_ARG, "sg_solve: restart must be 1..32");
  if (o.arith != SG_ARITH_F64 && o.arith != SG_ARITH_DF64 && o.arith != SG_ARITH_F64_DFOP)
    return sg_fail(h, SG_E_ARG, "sg_solve: bad arith");
  if (o.precond == SG_PC_BLOCKTRI_EXACT &&
      (o.method != SG_FGMRES || o.pc_prec != SG_F64 || o.arith != SG_ARITH_F64 || !(o.inner_tol >= 0) ||
       o.inner_restart < 0 || o.inner_restart > 32))
    return sg_fail(h, SG_E_ARG, "sg_solve: the exact block-triangular preconditioner needs FGMRES in FP64 "
                                "(pc_prec SG_F64, arith SG_ARITH_F64) and inner_restart <= 32");
  if (o.precond == SG_PC_BLOCKSYM_REC && (o.pc_prec != SG_F64 || o.arith != SG_ARITH_F64))
    return sg_fail(h, SG_E_ARG, "sg_solve: the recursive B_S is FP64 only (pc_prec SG_F64, arith SG_ARITH_F64)");
  if (h->elements == SG_P1 && (o.pc_prec != SG_F64 || o.arith != SG_ARITH_F64))
    return sg_fail(h, SG_E_ARG, "sg_solve: P1 elements solve in FP64 only (pc_prec SG_F64, arith SG_ARITH_F64)");
  h->inner_tol = o.inner_tol > 0 ? o.inner_tol : 1e-12;
  h->inner_restart = o.inner_restart > 0 ? o.inner_restart : 30;
  if (o.arith == SG_ARITH_DF64 && (o.method != SG_FGMRES || o.pc_prec == SG_F64))
    return sg_fail(h, SG_E_ARG, "sg_solve: double-float mode needs FGMRES with an FP32 or BF16 preconditioner");
  if (o.arith == SG_ARITH_F64_DFOP && ((o.method != SG_FGMRES && o.method != SG_GMRES) || o.pc_prec == SG_F64))
    return sg_fail(h, SG_E_ARG, "sg_solve: the double-float operator mode needs (F)GMRES with an FP32 or BF16 "
                                "preconditioner");
  sg_solve_info info{};
  const size_t N = h->Nx * (size_t)h->P;
  const bool dev = is_device_ptr(F) && is_device_ptr(U);
  const double* dF = F;
  double* dU = U;
  h->spec_dst = nullptr;
  h->spec_pending = false;
  if (!dev) {
    // FGMRES/GMRES copy the iterate early into page-locked U (overlapping the final residual check)
    if ((o.method == SG_GMRES || o.method == SG_FGMRES) && is_pinned_host(U)) h->spec_dst = U;
    if (!h->dstage && cudaMalloc(&h->dstage, sizeof(double) * N * 2) != cudaSuccess)
      return sg_fail(h, SG_E_ALLOC, "sg_solve: staging allocation");
    // cudaMemcpyDefault: one of F and U may be a device pointer (the runtime infers each direction)
    SG_CUDA(h, cudaMemcpyAsync(h->dstage, F, sizeof(double) * N, cudaMemcpyDefault, h->stream));
    dF = h->dstage;
    dU = h->dstage + N;
    if (o.x0_given) SG_CUDA(h, cudaMemcpyAsync(dU, U, sizeof(double) * N, cudaMemcpyDefault, h->stream));
  }
  cudaEvent_t e0, e1;
  SG_CUDA(h, cudaEventCreate(&e0));
  SG_CUDA(h, cudaEventCreate(&e1));
  SG_CUDA(h, cudaEventRecord(e0, h->stream));
  if (!o.x0_given) SG_CUDA(h, cudaMemsetAsync(dU, 0, sizeof(double) * N, h->stream));
  int rc;
  h->true_res_valid = false;
  if (o.method == SG_GMRES || o.method == SG_FGMRES) rc = solve_gmres(h, dF, dU, o, info, o.method == SG_FGMRES);
  else if (o.method == SG_GPCG) rc = solve_gpcg(h, dF, dU, o, info);
  else if (o.method == SG_PCG) rc = solve_pcg(h, dF, dU, o, info);
  else rc = solve_bgs(h, dF, dU, o, info);
  if ((rc == SG_OK && !h->true_res_valid) || rc == SG_E_NOCONV) {
    // true residual in FP64
    int rc2 = ensure_krylov(h, 1, 1, zprec_of(o.pc_prec));
    if (!rc2) rc2 = apply_f64(h,0, SG_F64, dU, SG_F64, h->ktmp, dF);
    double rr = 0, ff = 0;
    if (!rc2) rr = host_dot(h, h->ktmp, h->ktmp, N, &rc2);
    if (!rc2) ff = host_dot(h, dF, dF, N, &rc2);
    if (rc2) rc = rc2;
    else info.relres_true = ff > 0 ? std::sqrt(rr / ff) : 0.0;
  }
  if (!dev && (rc == SG_OK || rc == SG_E_NOCONV)) {
    if (rc == SG_OK && h->true_res_valid && h->spec_pending) {
      // the early copy holds the converged iterate: wait for it instead of copying again
      SG_CUDA(h, cudaStreamWaitEvent(h->stream, h->ev_c, 0));
    } else {
      int rc3 = spec_invalidate(h);
      if (rc3) return rc3;
      SG_CUDA(h, cudaMemcpyAsync(U, dU, sizeof(double) * N, cudaMemcpyDefault, h->stream));
    }
  } else if (h->spec_pending) {
    SG_CUDA(h, cudaStreamWaitEvent(h->stream, h->ev_c, 0));   // no copy in flight past the call
  }
  h->spec_dst = nullptr;
  h->spec_pending = false;
  SG_CUDA(h, cudaEventRecord(e1, h->stream));
  SG_CUDA(h, cudaEventSynchronize(e1));
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0), cudaEventDestroy(e1);
  info.t_total_ms = ms;
  info.status = rc;
  if (info_out) *info_out = info;
  return rc;
}

int sg_timing_enable(sg_handle h, int enable) {
  if (!h) return SG_E_ARG;
  if (const int rcd = sg_check_device(h, "sg_timing_enable")) return rcd;
  SG_CUDA(h, cudaStreamSynchronize(h->stream));
  for (auto& s : h->tr.spans) h->tr.pool.push_back(s.a), h->tr.pool.push_back(s.b);
  h->tr.spans.clear();
  for (auto& l : h->tr.launches) l = 0;
  h->tr.on = enable != 0;
  return SG_OK;
}

int sg_timing_read(sg_handle h, double* ms, long long* launches) {
  if (!h) return SG_E_ARG;
  if (const int rcd = sg_check_device(h, "sg_timing_read")) return rcd;
  SG_CUDA(h, cudaStreamSynchronize(h->stream));
  double acc[4] = {0, 0, 0, 0};
  for (auto& s : h->tr.spans) {
    float t = 0;
    if (cudaEventElapsedTime(&t, s.a, s.b) == cudaSuccess) acc[s.phase] += t;
    else cudaGetLastError();
    h->tr.pool.push_back(s.a), h->tr.pool.push_back(s.b);
  }
  h->tr.spans.clear();
  if (ms) std::copy(acc, acc + 4, ms);
  if (launches) std::copy(h->tr.launches, h->tr.launches + 4, launches);
  for (auto& l : h->tr.launches) l = 0;
  return SG_OK;
}

int sg_objective(sg_handle h, const double* U, double* J, double* G) {
  if (!h || !U || !J) return h ? sg_fail(h, SG_E_ARG, "sg_objective: null argument") : SG_E_ARG;
  if (const int rcd = sg_check_device(h, "sg_objective")) return rcd;
  std::vector<double> mu(h->P);
  int rc = objective_dots(h, U, mu.data());
  if (rc) return rc;
  double j = mu[0];
  for (int i = 1; i < h->P; ++i) j += 0.5 * mu[i] * mu[i];
  *J = j;
  if (G) {
    if ((rc = objective_grad(h, h->pvec, G))) return rc;
    SG_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  return SG_OK;
}

int sg_adjoint_gradients(sg_handle h, const double* U, const double* Lam, double sigma, double* g_abar, double* g_sigma) {
  if (!h || !U || !Lam) return h ? sg_fail(h, SG_E_ARG, "sg_adjoint_gradients: null argument") : SG_E_ARG;
  if (h->elements != SG_Q1) return sg_fail(h, SG_E_ARG, "sg_adjoint_gradients: Q1 elements only");
  if (const int rcd = sg_check_device(h, "sg_adjoint_gradients")) return rcd;
  int rc;
  if (g_abar && (rc = adj_cell_forms(h, U, Lam, g_abar))) return rc;
  if (g_sigma) {
    if (!(sigma != 0.0)) return sg_fail(h, SG_E_ARG, "sg_adjoint_gradients: sigma must be nonzero");
    if ((rc = ensure_krylov(h, 1, 1, SG_F64))) return rc;
    // (A - I (x) K_0) U = sum_{k>=1} G_k (x) K_k U, linear in sigma
    if ((rc = apply_f64(h,3, SG_F64, U, SG_F64, h->ktmp, nullptr))) return rc;
    const double d = host_dot(h, Lam, h->ktmp, h->Nx * (size_t)h->P, &rc);
    if (rc) return rc;
    *g_sigma = -d / sigma;
  }
  SG_CUDA(h, cudaStreamSynchronize(h->stream));
  return SG_OK;
}

}  // extern "C"
