// Batched solves in one CUDA graph: every system's restarted flexible GMRES (Sec. 4.2, 6) with its
// Arnoldi control on the device, all systems as parallel branches of one graph, one graph launch per
// restart cycle of the whole batch.
//
// Per system the graph holds a chain
//     begin -> IF(c_0){ step 0 } -> IF(c_1){ step 1 } -> ... -> IF(c_{m-1}){ step m-1 } -> IF(c_t){ tail }
// begin reads the squared norm of the current residual (stored, unnormalised, as v_0), decides
// whether the system has converged, failed or ran out of iterations, and opens c_0 and c_t; step j is
// the preconditioner, the grid maxima of z_j, the operator, the Gram-Schmidt dots, a one-thread kernel
// that scales the coefficients, the Gram-Schmidt update with its norm, and a one-thread kernel that
// forms the Hessenberg column, applies and extends the Givens rotations and opens c_{j+1} unless the
// residual estimate has met the tolerance (or the step budget or a breakdown ends the cycle); the
// tail solves the triangular system, updates U, recomputes the FP64 true residual into v_0 and its
// norm.  Conditional handles default to 0 at every launch, so a closed step closes every later one.
// All systems run concurrently; the host launches the graph again while any system is still running,
// and reads the outcome once per launch.  The arithmetic is that of sg_solve's FGMRES with the FP64
// basis (SG_ARITH_F64 or SG_ARITH_F64_DFOP), step by step, with the host's scalar work done by the
// one-thread kernels in FP64.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "df64.cuh"
#include "sg_internal.h"
#include "update_q.cuh"

namespace {

// Device-side state of one system's FGMRES (one per handle).
struct GDev {
  double H[(SG_MAX_RESTART + 1) * SG_MAX_RESTART];
  double cs[SG_MAX_RESTART], sn[SG_MAX_RESTART], g[SG_MAX_RESTART + 1], sc[SG_MAX_RESTART + 1];
  double y[SG_MAX_RESTART];
  double bnorm, tol, rr, relres_est, relres_true;
  int k, its, maxit, m, status, cycles;
};
constexpr int GS_RUNNING = 1;        // status while the solve goes on (final statuses are sg_status codes)

// after the initial norm (slot 0 of the reductions holds ||F||^2 = ||v_0||^2)
__global__ void k_g_init(GDev* d, const double* red, double tol, int maxit, int m) {
  const double bb = red[0];
  d->bnorm = sqrt(bb);
  d->rr = bb;
  d->tol = tol;
  d->maxit = maxit;
  d->m = m;
  d->its = 0;
  d->k = 0;
  d->cycles = 0;
  d->relres_est = d->relres_true = 0.0;
  d->status = isfinite(bb) ? (bb == 0.0 ? SG_OK : GS_RUNNING) : SG_E_NONFINITE;
}

__global__ void k_g_begin(GDev* d, cudaGraphConditionalHandle c0, cudaGraphConditionalHandle ct) {
  d->k = 0;
  if (d->status != GS_RUNNING) return;
  const double beta = sqrt(d->rr);
  if (!isfinite(beta)) {
    d->status = SG_E_NONFINITE;
    return;
  }
  d->relres_true = beta / d->bnorm;
  if (beta <= d->tol * d->bnorm) {
    d->relres_est = d->relres_true;
    d->status = SG_OK;
    return;
  }
  if (d->its >= d->maxit) {
    d->status = SG_E_NOCONV;
    return;
  }
  for (int i = 0; i <= d->m; ++i) d->g[i] = 0.0;
  d->g[0] = beta;
  d->sc[0] = 1.0 / beta;
  cudaGraphSetConditional(c0, 1);
  cudaGraphSetConditional(ct, 1);
}

// Gram-Schmidt coefficients of the stored (lazily normalised) basis: coef_i = s_i^2 (V^T w)_i
__global__ void k_g_coef(const GDev* d, const double* red, double* coef, int j) {
  for (int i = threadIdx.x; i <= j; i += blockDim.x) coef[i] = d->sc[i] * d->sc[i] * red[i];
}

// Hessenberg column j, Givens rotations, residual estimate; opens step j + 1 when it is to run
__global__ void k_g_givens(GDev* d, const double* dv, const double* nrm, int j, cudaGraphConditionalHandle cn,
                           int has_next) {
  const int m = d->m;
  double* H = d->H;
  const double nrm2 = nrm[0];
  const double hn = d->sc[j] * sqrt(nrm2);
  for (int i = 0; i <= j; ++i) {
    const double hij = d->sc[i] * d->sc[j] * dv[i];
    if (!isfinite(hij)) {
      d->status = SG_E_NONFINITE;
      return;
    }
    H[i * m + j] = hij;
  }
  if (!isfinite(hn)) {
    d->status = SG_E_NONFINITE;
    return;
  }
  H[(j + 1) * m + j] = hn;
  for (int i = 0; i < j; ++i) {
    const double t = d->cs[i] * H[i * m + j] + d->sn[i] * H[(i + 1) * m + j];
    H[(i + 1) * m + j] = -d->sn[i] * H[i * m + j] + d->cs[i] * H[(i + 1) * m + j];
    H[i * m + j] = t;
  }
  const double dd = hypot(H[j * m + j], H[(j + 1) * m + j]);
  if (dd == 0.0) {
    d->status = SG_E_BREAKDOWN;
    return;
  }
  d->cs[j] = H[j * m + j] / dd;
  d->sn[j] = H[(j + 1) * m + j] / dd;
  H[j * m + j] = dd;
  H[(j + 1) * m + j] = 0.0;
  d->g[j + 1] = -d->sn[j] * d->g[j];
  d->g[j] = d->cs[j] * d->g[j];
  d->its += 1;
  d->k = j + 1;
  d->relres_est = fabs(d->g[j + 1]) / d->bnorm;
  if (hn == 0.0 || fabs(d->g[j + 1]) <= d->tol * d->bnorm || d->its >= d->maxit || !has_next) return;
  d->sc[j + 1] = 1.0 / sqrt(nrm2);
  cudaGraphSetConditional(cn, 1);
}

// back substitution H y = g over the k steps of the cycle, y_i scaled by s_i (the stored z_i are z_i / s_i);
// no update after a failure
__global__ void k_g_backsub(GDev* d) {
  const int m = d->m;
  int k = d->k;
  if (d->status != GS_RUNNING) k = d->k = 0;
  for (int i = k - 1; i >= 0; --i) {
    double s = d->g[i];
    for (int l = i + 1; l < k; ++l) s -= d->H[i * m + l] * d->y[l];
    d->y[i] = s / d->H[i * m + i];
  }
  for (int i = 0; i < k; ++i) d->y[i] *= d->sc[i];
}

// after the true residual's norm (slot 0)
__global__ void k_g_end(GDev* d, const double* red) {
  const double rr = red[0];
  d->rr = rr;
  d->cycles += 1;
  if (d->status != GS_RUNNING) return;
  const double rel = sqrt(rr) / d->bnorm;
  d->relres_true = rel;
  if (!isfinite(rel)) d->status = SG_E_NONFINITE;
  else if (rel <= d->tol) d->relres_est = rel, d->status = SG_OK;
}

// U += sum_{l < k} y_l z'_l for the FP32 z_l read through their grids (SG_F32Q); y and k on the device
template <int NV>
__global__ void k_g_update_q(double* __restrict__ U, const float* __restrict__ Z, size_t ldz, const GDev* d, int c0,
                             size_t Nx, const unsigned* __restrict__ qmax, int P) {
  const int b = blockIdx.y;
  const int nz = min(d->k - c0, NV);
  if (nz <= 0) return;
  // per column: y_l as double-float, the block's grid scale and quantum (zero past nz), once per CTA in
  // shared memory; every column load is issued before the sums (slots past nz re-read the last column)
  __shared__ float4 kc[NV];
  for (int l = threadIdx.x; l < NV; l += blockDim.x) {
    const df2 c = df_from_double(l < nz ? d->y[c0 + l] : 0.0);
    const unsigned mb = l < nz ? qmax[(size_t)(c0 + l) * P + b] : 0u;
    kc[l] = make_float4(c.hi, c.lo, qgrid_scale(mb), qgrid_quantum(mb));
  }
  __syncthreads();
  update_q_block<NV>(U, Z + (size_t)c0 * ldz, ldz, kc, nz, Nx, b);
}

// U += sum_{l < k} y_l z_l for z_l stored in TZ
template <typename TZ, int NV>
__global__ void k_g_update(double* __restrict__ U, const TZ* __restrict__ Z, size_t ldz, const GDev* d, int c0,
                           size_t N) {
  const int nz = min(d->k - c0, NV);
  if (nz <= 0) return;
  const TZ* Zc = Z + (size_t)c0 * ldz;
  if constexpr (sizeof(TZ) == 8) {
    double c[NV];
#pragma unroll
    for (int l = 0; l < NV; ++l) c[l] = (l < nz) ? d->y[c0 + l] : 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
      double u = U[i];
#pragma unroll
      for (int l = 0; l < NV; ++l)
        if (l < nz) u += c[l] * ld_as<double>(Zc + (size_t)l * ldz + i);
      U[i] = u;
    }
  } else {                       // as k_update: the sum in double-float, one FP64 addition
    __shared__ float2 kc[NV];
    for (int l = threadIdx.x; l < NV; l += blockDim.x) {
      const df2 c = df_from_double(l < nz ? d->y[c0 + l] : 0.0);
      kc[l] = make_float2(c.hi, c.lo);
    }
    __syncthreads();
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
      float zv[NV];
#pragma unroll
      for (int l = 0; l < NV; ++l) zv[l] = ld_as<float>(Zc + (size_t)min(l, nz - 1) * ldz + i);
      const double u0 = U[i];
      dacc a = dacc_zero();
#pragma unroll
      for (int l = 0; l < NV; ++l) {
        const float2 k = kc[l];
        dacc_fma(a, df2{k.x, k.y}, zv[l]);
      }
      const df2 r = dacc_get(a);
      U[i] = (u0 + (double)r.hi) + (double)r.lo;
    }
  }
}

struct GSys {
  sg_ctx* h;
  const double* F;
  double* U;
  GDev* d = nullptr;
  cudaStream_t saved = nullptr;
};

int grid_x(size_t N) { return (int)std::max<size_t>(1, std::min<size_t>((N + 4095) / 4096, 64)); }

// the vector and scalar launches of one system, on h->stream (captured into the batch graph)
struct GSteps {
  GSys& s;
  const sg_solve_opts& o;
  sg_ctx* h() const { return s.h; }
  size_t Np() const { return s.h->Np; }
  size_t N() const { return s.h->Nx * (size_t)s.h->P; }
  int zp() const { return zprec_of(o.pc_prec); }
  bool quant() const { return o.arith == SG_ARITH_F64_DFOP && zp() == SG_F32; }
  double* v(int l) const { return s.h->kv + Np() * l; }
  void* z(int j) const { return (char*)s.h->kz + prec_size(zp()) * Np() * j; }
  unsigned* qm(int j) const { return s.h->qmax + (size_t)j * s.h->P; }

  int step(int j, cudaGraphConditionalHandle cn, bool has_next) {
    sg_ctx* H = h();
    int rc;
    H->zmax_out = quant() ? qm(j) : nullptr;
    H->zmax_done = false;
    rc = apply_precond_ext(H, o.precond, SG_F64, v(j), z(j), o.pc_prec, o.transpose);
    H->zmax_out = nullptr;
    if (rc) return rc;
    if (quant() && !H->zmax_done && (rc = block_absmax(H, (const float*)z(j), qm(j)))) return rc;
    H->qcur = quant() ? qm(j) : nullptr;
    const int arith = o.arith == SG_ARITH_F64_DFOP ? SG_DF64 : SG_F64;
    if ((rc = launch_apply(H, 0, quant() ? SG_F32Q : zp(), z(j), 0, SG_F64, v(j + 1), 0, SG_F64, nullptr, 0, 0, H->P, 0,
                           0, arith)))
      return rc;
    if ((rc = vec_dots(H, H->kv, Np(), j + 1, v(j + 1), Np(), true, nullptr))) return rc;
    double* coef = const_cast<double*>(red_slot(H, 3));
    k_g_coef<<<1, 64, 0, H->stream>>>(s.d, red_slot(H, 0), coef, j);
    SG_CUDA(H, cudaGetLastError());
    if ((rc = vec_axpys_norm(H, H->kv, Np(), j + 1, coef, v(j + 1), Np(), nullptr))) return rc;
    k_g_givens<<<1, 1, 0, H->stream>>>(s.d, red_slot(H, 0), red_slot(H, 1), j, cn, has_next ? 1 : 0);
    SG_CUDA(H, cudaGetLastError());
    count_launch(H, 2);
    return SG_OK;
  }

  int tail() {
    sg_ctx* H = h();
    int rc;
    k_g_backsub<<<1, 1, 0, H->stream>>>(s.d);
    SG_CUDA(H, cudaGetLastError());
    for (int c0 = 0; c0 < o.restart; c0 += 16) {
      if (quant())
        k_g_update_q<16><<<dim3(grid_x(H->Nx), H->P), 256, 0, H->stream>>>(s.U, (const float*)H->kz, Np(), s.d, c0,
                                                                            H->Nx, H->qmax, H->P);
      else if (zp() == SG_F64)
        k_g_update<double, 16><<<grid_x(N()), 256, 0, H->stream>>>(s.U, (const double*)H->kz, Np(), s.d, c0, N());
      else if (zp() == SG_F32)
        k_g_update<float, 16><<<grid_x(N()), 256, 0, H->stream>>>(s.U, (const float*)H->kz, Np(), s.d, c0, N());
      else
        k_g_update<bf16, 16><<<grid_x(N()), 256, 0, H->stream>>>(s.U, (const bf16*)H->kz, Np(), s.d, c0, N());
      SG_CUDA(H, cudaGetLastError());
    }
    // the IEEE FP64 true residual into the stored v_0 and its squared norm
    if ((rc = launch_apply(H, 0, SG_F64, s.U, 0, SG_F64, v(0), 0, SG_F64, s.F, 0, 0, H->P, 0, 0, SG_F64))) return rc;
    if ((rc = vec_dots(H, H->kv, Np(), 0, v(0), Np(), true, nullptr))) return rc;
    k_g_end<<<1, 1, 0, H->stream>>>(s.d, red_slot(H, 0));
    SG_CUDA(H, cudaGetLastError());
    count_launch(H, 2 + (o.restart + 15) / 16);
    return SG_OK;
  }
};

// appends a conditional IF node after dep and captures its body from the system's launches
template <class Body>
int add_if(sg_ctx* h, cudaGraph_t G, cudaGraphNode_t* dep, cudaGraphConditionalHandle c, Body&& body) {
  cudaGraphNodeParams p{};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = c;
  p.conditional.type = cudaGraphCondTypeIf;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  SG_CUDA(h, cudaGraphAddNode(&node, G, dep, nullptr, dep ? 1 : 0, &p));
  cudaGraph_t bodyg = p.conditional.phGraph_out[0];
  SG_CUDA(h, cudaStreamBeginCaptureToGraph(h->stream, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  const int rc = body();
  cudaGraph_t out = nullptr;
  const cudaError_t e = cudaStreamEndCapture(h->stream, &out);
  if (rc) return rc;
  if (e != cudaSuccess) return sg_fail(h, SG_E_CUDA, std::string("batch graph: body capture: ") + cudaGetErrorString(e));
  *dep = node;
  return SG_OK;
}

// captures a launch sequence directly into G (after dep, when given) and leaves in *dep the node the
// sequence ends with
template <class Body>
int add_plain(sg_ctx* h, cudaGraph_t G, cudaGraphNode_t* dep, Body&& body) {
  SG_CUDA(h, cudaStreamBeginCaptureToGraph(h->stream, G, *dep ? dep : nullptr, nullptr, *dep ? 1 : 0,
                                           cudaStreamCaptureModeThreadLocal));
  int rc = body();
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  if (!rc && (cudaStreamGetCaptureInfo(h->stream, &st, nullptr, nullptr, &deps, nullptr, &nd) != cudaSuccess || nd != 1))
    rc = sg_fail(h, SG_E_CUDA, "batch graph: capture did not end in one node");
  const cudaGraphNode_t last = (!rc && deps) ? deps[0] : nullptr;
  cudaGraph_t out = nullptr;
  const cudaError_t e = cudaStreamEndCapture(h->stream, &out);
  if (rc) return rc;
  if (e != cudaSuccess) return sg_fail(h, SG_E_CUDA, std::string("batch graph: capture: ") + cudaGetErrorString(e));
  *dep = last;
  return SG_OK;
}
}  // namespace

// A built batch: the systems, the options, and two instantiated graphs -- the start (U = 0, v_0 = F, its
// norm, the device state) and one restart cycle of every system.
struct sg_batch_ctx {
  std::vector<GSys> sys;
  sg_solve_opts o{};
  cudaStream_t cs = nullptr;
  cudaGraphExec_t Xs = nullptr, Xc = nullptr;
  std::vector<const void*> ws;      // the workspace pointers the graphs were captured with
  std::string err;
};

namespace {
std::vector<const void*> workspace_of(const sg_batch_ctx* b) {
  std::vector<const void*> w;
  for (const auto& g : b->sys) {
    const sg_ctx* h = g.h;
    w.insert(w.end(), {h->kv, h->kz, h->qmax, h->red_out, h->red_partial, h->red_count, h->ktmp});
    for (const auto& W : h->work) {
      w.insert(w.end(), {W.T, W.T32, W.S1, W.S2});
      for (int l = 0; l < SG_MAX_LEVELS; ++l) w.insert(w.end(), {W.b[l], W.x[l]});
    }
  }
  return w;
}

void batch_free(sg_batch_ctx* b) {
  if (!b) return;
  if (b->Xs) cudaGraphExecDestroy(b->Xs);
  if (b->Xc) cudaGraphExecDestroy(b->Xc);
  for (auto& g : b->sys) {
    if (g.d) cudaFree(g.d);
    if (g.h) g.h->stream = g.saved;
  }
  if (b->cs) cudaStreamDestroy(b->cs);
  delete b;
}

int batch_build(sg_batch_ctx* b) {
  const sg_solve_opts& o = b->o;
  sg_ctx* h0 = b->sys[0].h;
  int rc = SG_OK;
  // workspaces, and one preconditioner application outside any capture (it allocates what it needs)
  for (auto& g : b->sys) {
    sg_ctx* h = g.h;
    h->stream = b->cs;
    if ((rc = ensure_krylov_ext(h, o.restart + 1, o.restart, zprec_of(o.pc_prec), 0))) return rc;
    if (o.precond != SG_PC_NONE && (rc = ensure_prec_work(h, o.pc_prec))) return rc;
    if ((rc = apply_precond_ext(h, o.precond, SG_F64, g.F, h->kz, o.pc_prec, o.transpose))) return rc;
    if (cudaMalloc(&g.d, sizeof(GDev)) != cudaSuccess) return sg_fail(h, SG_E_ALLOC, "batch: device state");
  }
  SG_CUDA(h0, cudaStreamSynchronize(b->cs));
  // the start graph
  cudaGraph_t S = nullptr, C = nullptr;
  SG_CUDA(h0, cudaGraphCreate(&S, 0));
  for (auto& g : b->sys) {
    if (rc) break;
    sg_ctx* h = g.h;
    cudaGraphNode_t dep = nullptr;
    rc = add_plain(h, S, &dep, [&]() -> int {
      const size_t N = h->Nx * (size_t)h->P;
      SG_CUDA(h, cudaMemsetAsync(g.U, 0, sizeof(double) * N, h->stream));
      SG_CUDA(h, cudaMemcpyAsync(h->kv, g.F, sizeof(double) * N, cudaMemcpyDeviceToDevice, h->stream));
      int r = vec_dots(h, h->kv, h->Np, 0, h->kv, h->Np, true, nullptr);
      if (r) return r;
      k_g_init<<<1, 1, 0, h->stream>>>(g.d, red_slot(h, 0), o.tol, o.maxit, o.restart);
      SG_CUDA(h, cudaGetLastError());
      return SG_OK;
    });
  }
  // the cycle graph: one chain of conditional steps per system, the chains side by side
  if (!rc && cudaGraphCreate(&C, 0) != cudaSuccess) rc = sg_fail(h0, SG_E_CUDA, "batch: graph");
  for (auto& g : b->sys) {
    if (rc) break;
    sg_ctx* h = g.h;
    const int m = o.restart;
    std::vector<cudaGraphConditionalHandle> c(m + 1);
    for (int j = 0; j <= m && !rc; ++j)
      if (cudaGraphConditionalHandleCreate(&c[j], C, 0, cudaGraphCondAssignDefault) != cudaSuccess)
        rc = sg_fail(h, SG_E_CUDA, "batch: conditional handle");
    if (rc) break;
    GSteps st{g, o};
    cudaGraphNode_t dep = nullptr;
    rc = add_plain(h, C, &dep, [&]() -> int {
      k_g_begin<<<1, 1, 0, h->stream>>>(g.d, c[0], c[m]);
      SG_CUDA(h, cudaGetLastError());
      count_launch(h);
      return SG_OK;
    });
    for (int j = 0; j < m && !rc; ++j)
      rc = add_if(h, C, &dep, c[j], [&]() -> int { return st.step(j, c[j + 1 < m ? j + 1 : j], j + 1 < m); });
    if (!rc) rc = add_if(h, C, &dep, c[m], [&]() -> int { return st.tail(); });
  }
  if (!rc) {
    cudaError_t e = cudaGraphInstantiate(&b->Xs, S, 0);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->Xc, C, 0);
    if (e != cudaSuccess) rc = sg_fail(h0, SG_E_CUDA, std::string("batch: instantiate: ") + cudaGetErrorString(e));
  }
  if (S) cudaGraphDestroy(S);
  if (C) cudaGraphDestroy(C);
  b->ws = workspace_of(b);
  return rc;
}
}  // namespace

extern "C" int sg_batch_create(sg_handle* hs, const double* const* F, double* const* U, int nsys,
                               const sg_solve_opts* opts, sg_batch* out) {
  if (!out) return SG_E_ARG;
  *out = nullptr;
  if (!hs || !F || !U || !opts || nsys < 1) return SG_E_ARG;
  for (int s = 0; s < nsys; ++s)
    if (!hs[s] || !F[s] || !U[s]) return SG_E_ARG;
  {
    std::vector<sg_handle> seen(hs, hs + nsys);
    std::sort(seen.begin(), seen.end());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) return SG_E_ARG;
  }
  const sg_solve_opts o = *opts;
  sg_ctx* h0 = hs[0];
  for (int s = 0; s < nsys; ++s)
    if (const int rcd = sg_check_device(hs[s], "sg_batch_create")) return rcd;
  if (o.method != SG_FGMRES || (o.arith != SG_ARITH_F64 && o.arith != SG_ARITH_F64_DFOP) || o.restart < 1 ||
      o.restart > 32 || o.x0_given || o.reorth || !(o.tol > 0) || o.maxit < 0 || o.precond < 0 || o.precond > 3 ||
      o.pc_prec < 0 || o.pc_prec > 4 || o.pc_prec == SG_DF64 || (o.arith == SG_ARITH_F64_DFOP && o.pc_prec == SG_F64))
    return sg_fail(h0, SG_E_ARG, "batch graph: FGMRES with an FP64 basis (arith SG_ARITH_F64, or SG_ARITH_F64_DFOP "
                                 "with a low-precision preconditioner), restart 1..32, no initial guess, no "
                                 "reorthogonalisation");
  sg_batch_ctx* b = new sg_batch_ctx();
  b->o = o;
  for (int s = 0; s < nsys; ++s) {
    GSys g{};
    g.h = hs[s], g.F = F[s], g.U = U[s], g.saved = hs[s]->stream;
    b->sys.push_back(g);
  }
  if (cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking) != cudaSuccess) {
    b->cs = nullptr;
    batch_free(b);
    return sg_fail(h0, SG_E_CUDA, "batch: stream");
  }
  const int rc = batch_build(b);
  for (auto& g : b->sys) g.h->stream = g.saved;
  if (rc) {
    batch_free(b);
    return rc;
  }
  *out = b;
  return SG_OK;
}

extern "C" int sg_batch_solve(sg_batch b, sg_solve_info* infos) {
  if (!b) return SG_E_ARG;
  sg_ctx* h0 = b->sys[0].h;
  if (workspace_of(b) != b->ws)
    return sg_fail(h0, SG_E_STATE, "sg_batch_solve: a handle's workspace changed since sg_batch_create; rebuild the batch");
  for (auto& g : b->sys)
    if (const int rcd = sg_check_device(g.h, "sg_batch_solve")) return rcd;
  const int nsys = (int)b->sys.size();
  // one launch of the start graph, then one launch of the cycle graph per restart cycle while a system runs
  SG_CUDA(h0, cudaGraphLaunch(b->Xs, b->cs));
  const int max_launch = (b->o.maxit + b->o.restart - 1) / b->o.restart + 2;
  std::vector<GDev> host(nsys);
  for (int launch = 0; launch < max_launch; ++launch) {
    SG_CUDA(h0, cudaGraphLaunch(b->Xc, b->cs));
    for (int s = 0; s < nsys; ++s)
      SG_CUDA(h0, cudaMemcpyAsync(&host[s], b->sys[s].d, sizeof(GDev), cudaMemcpyDeviceToHost, b->cs));
    SG_CUDA(h0, cudaStreamSynchronize(b->cs));
    bool running = false;
    for (int s = 0; s < nsys; ++s) running = running || host[s].status == GS_RUNNING;
    if (!running) break;
  }
  int first_err = SG_OK;
  for (int s = 0; s < nsys; ++s) {
    const GDev& d = host[s];
    const int st = d.status == GS_RUNNING ? SG_E_NOCONV : d.status;
    if (infos) {
      sg_solve_info in{};
      in.iters = d.its;
      in.restarts = d.cycles > 0 ? d.cycles - 1 : 0;
      in.status = st;
      in.relres_est = d.relres_est;
      in.relres_true = d.relres_true;
      infos[s] = in;
    }
    if (st != SG_OK && first_err == SG_OK) first_err = st;
  }
  return first_err;
}

extern "C" void sg_batch_destroy(sg_batch b) {
  if (b && b->cs) cudaStreamSynchronize(b->cs);
  batch_free(b);
}

extern "C" int sg_solve_batch_graph(sg_handle* hs, const double* const* F, double* const* U, int nsys,
                                    const sg_solve_opts* opts, sg_solve_info* infos) {
  if (nsys == 0 && hs && F && U && opts) return SG_OK;
  sg_batch b = nullptr;
  int rc = sg_batch_create(hs, F, U, nsys, opts, &b);
  if (rc) return rc;
  rc = sg_batch_solve(b, infos);
  sg_batch_destroy(b);
  return rc;
}
