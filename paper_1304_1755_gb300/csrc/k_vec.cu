// FP64 Krylov vector kernels: fused multi-dot (Arnoldi h = V^T w), fused
// multi-axpy with norm (w -= V h, ||w||^2), scaling, solution updates, casts and
// the small fused updates of GPCG[1] / PCG (Sec. 4.2).  Reductions are
// deterministic: warp shuffles, a per-block partial in global memory and a
// fixed-order sum by the last block to finish.
#include <algorithm>
#include <vector>

#include "sg_internal.h"

namespace {
constexpr int NT = SG_NTHREADS_RED;
constexpr int MAXOUT = 40;

template <int NO>
__device__ __forceinline__ void reduce_out(double (&acc)[NO], double* partial, double* out, unsigned* counter, int nout) {
  __shared__ double red[NT / 32][NO];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 0; o < NO; ++o) {
    double v = acc[o];
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    if (lane == 0) red[warp][o] = v;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < nout; o += blockDim.x) {
    double v = 0;
    for (int w = 0; w < NT / 32; ++w) v += red[w][o];
    partial[(size_t)blockIdx.x * MAXOUT + o] = v;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (last) {
    __threadfence();
    for (int o = threadIdx.x; o < nout; o += blockDim.x) {
      double v = 0;
      for (int b = 0; b < (int)gridDim.x; ++b) v += ((volatile double*)partial)[(size_t)b * MAXOUT + o];
      out[o] = v;
    }
    if (threadIdx.x == 0) *counter = 0u;
  }
}

template <int NV>
__global__ void __launch_bounds__(NT) k_dots(const double* __restrict__ V, size_t ldv, int nv,
                                             const double* __restrict__ w, size_t N, int with_ww, double* partial,
                                             double* out, unsigned* counter) {
  double acc[NV + 1];
#pragma unroll
  for (int l = 0; l <= NV; ++l) acc[l] = 0;
  for (size_t s = blockIdx.x * (size_t)NT + threadIdx.x; s < N; s += (size_t)gridDim.x * NT) {
    const double wv = w[s];
#pragma unroll
    for (int l = 0; l < NV; ++l)
      if (l < nv) acc[l] += V[(size_t)l * ldv + s] * wv;
    acc[NV] += wv * wv;
  }
  // move the w.w slot next to the last used one
  double tmp[NV + 1];
#pragma unroll
  for (int l = 0; l <= NV; ++l) tmp[l] = (l < nv) ? acc[l] : (l == nv ? acc[NV] : 0.0);
  reduce_out<NV + 1>(tmp, partial, out, counter, nv + (with_ww ? 1 : 0));
}

template <int NV>
__global__ void __launch_bounds__(NT) k_axpys(const double* __restrict__ V, size_t ldv, int nv,
                                              const double* __restrict__ hc, double* __restrict__ w, size_t N,
                                              double* partial, double* out, unsigned* counter) {
  double c[NV];
#pragma unroll
  for (int l = 0; l < NV; ++l) c[l] = (l < nv) ? hc[l] : 0.0;
  double acc[1] = {0};
  for (size_t s = blockIdx.x * (size_t)NT + threadIdx.x; s < N; s += (size_t)gridDim.x * NT) {
    double v = w[s];
#pragma unroll
    for (int l = 0; l < NV; ++l)
      if (l < nv) v -= c[l] * V[(size_t)l * ldv + s];
    w[s] = v;
    acc[0] += v * v;
  }
  reduce_out<1>(acc, partial, out, counter, 1);
}

__global__ void k_scale(const double* __restrict__ w, double* __restrict__ v, size_t N, double s) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    v[i] = w[i] * s;
}

template <typename TZ, int NV>
__global__ void k_update(double* __restrict__ U, const TZ* __restrict__ Z, size_t ldz, int nz,
                         const double* __restrict__ y, size_t N) {
  double c[NV];
#pragma unroll
  for (int l = 0; l < NV; ++l) c[l] = (l < nz) ? y[l] : 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    double u = U[i];
#pragma unroll
    for (int l = 0; l < NV; ++l)
      if (l < nz) u += c[l] * ld_as<double>(Z + (size_t)l * ldz + i);
    U[i] = u;
  }
}

template <typename TI, typename TO>
__global__ void k_cast(const TI* __restrict__ in, TO* __restrict__ out, size_t N) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    st_as<TO, double>(out + i, ld_as<double>(in + i));
}

__global__ void k_axpby(double a, const double* __restrict__ x, double b, double* __restrict__ y, size_t N) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

template <typename TX>
__global__ void k_axpy_prec(double a, const TX* __restrict__ x, double* __restrict__ y, size_t N) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    y[i] += a * ld_as<double>(x + i);
}

// up to 4 dot products <x_q, y_q> in one pass; y_q in any storage precision
struct DotPairs {
  const double* x[4];
  const void* y[4];
  int yp[4];
  int n;
};
__device__ __forceinline__ double ld_any(const void* p, int prec, size_t i) {
  if (prec == SG_F64) return ((const double*)p)[i];
  if (prec == SG_F32) return (double)((const float*)p)[i];
  return (double)__bfloat162float(((const bf16*)p)[i]);
}
__global__ void __launch_bounds__(NT) k_dotpairs(DotPairs D, size_t N, double* partial, double* out, unsigned* counter) {
  double acc[4] = {0, 0, 0, 0};
  for (size_t s = blockIdx.x * (size_t)NT + threadIdx.x; s < N; s += (size_t)gridDim.x * NT) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (q < D.n) acc[q] += D.x[q][s] * ld_any(D.y[q], D.yp[q], s);
  }
  reduce_out<4>(acc, partial, out, counter, D.n);
}

// per cell e: -sum_i Lam_i|e^T K_ref U_i|e  (adjoint gradient w.r.t. abar_e)
__global__ void k_cell_forms(const double* __restrict__ U, const double* __restrict__ L, double* __restrict__ g,
                             int n, int m, int P, size_t Nx) {
  const size_t Nc = (size_t)(n - 1) * (n - 1);
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < Nc; e += (size_t)gridDim.x * blockDim.x) {
    const int cx = (int)(e % (n - 1)), cy = (int)(e / (n - 1));
    const int vx[4] = {cx, cx + 1, cx + 1, cx}, vy[4] = {cy, cy, cy + 1, cy + 1};
    long idx[4];
    for (int a = 0; a < 4; ++a)
      idx[a] = (vx[a] >= 1 && vx[a] <= n - 2 && vy[a] >= 1 && vy[a] <= n - 2) ? (long)(vx[a] - 1) + (long)(vy[a] - 1) * m : -1;
    double s = 0;
    for (int i = 0; i < P; ++i) {
      double u[4], l[4];
      for (int a = 0; a < 4; ++a) {
        u[a] = idx[a] >= 0 ? U[(size_t)i * Nx + idx[a]] : 0.0;
        l[a] = idx[a] >= 0 ? L[(size_t)i * Nx + idx[a]] : 0.0;
      }
      // K_ref = (1/2) f1 f1^T + (1/2) f2 f2^T + (1/6) f3 f3^T
      const double du1 = u[0] - u[2], du2 = u[1] - u[3], du3 = u[0] - u[1] + u[2] - u[3];
      const double dl1 = l[0] - l[2], dl2 = l[1] - l[3], dl3 = l[0] - l[1] + l[2] - l[3];
      s += 0.5 * (dl1 * du1 + dl2 * du2) + dl3 * du3 / 6.0;
    }
    g[e] = -s;
  }
}

// mu_i = m^T U_i with m_s = h^2 (one block per PC row)
__global__ void k_row_sums(const double* __restrict__ U, size_t Nx, double h2, double* __restrict__ mu) {
  __shared__ double red[NT / 32];
  const double* u = U + (size_t)blockIdx.x * Nx;
  double acc = 0;
  for (size_t s = threadIdx.x; s < Nx; s += blockDim.x) acc += u[s];
  for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) v += red[w];
    mu[blockIdx.x] = h2 * v;
  }
}

// G_0 = m, G_i = mu_i m (i >= 1)
__global__ void k_obj_grad(const double* __restrict__ mu, double* __restrict__ G, size_t Nx, int P, double h2) {
  const size_t N = Nx * (size_t)P;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < N; t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / Nx);
    G[t] = (i == 0 ? 1.0 : mu[i]) * h2;
  }
}

int grid_for(size_t N) {
  size_t b = (N + 255) / 256;
  return (int)std::max<size_t>(1, std::min<size_t>(b, 152 * 16));
}
}  // namespace

int ensure_reduction(sg_ctx* h) {
  if (h->red_partial) return SG_OK;
  h->red_blocks = 152 * 4;
  if (cudaMalloc(&h->red_partial, sizeof(double) * MAXOUT * h->red_blocks) != cudaSuccess ||
      cudaMalloc(&h->red_out, sizeof(double) * 4 * MAXOUT) != cudaSuccess ||
      cudaMalloc(&h->red_count, sizeof(unsigned) * 8) != cudaSuccess ||
      cudaMallocHost(&h->red_host, sizeof(double) * 4 * MAXOUT) != cudaSuccess)
    return sg_fail(h, SG_E_ALLOC, "alloc reduction buffers");
  SG_CUDA(h, cudaMemsetAsync(h->red_count, 0, sizeof(unsigned) * 8, h->stream));
  return SG_OK;
}

static int red_grid(sg_ctx* h, size_t N) {
  return (int)std::max<size_t>(1, std::min<size_t>((size_t)h->red_blocks, (N + NT - 1) / NT));
}

// h[0..nv) = V^T w (and w.w in slot nv when with_ww), result left in red_out[0..] on the device and,
// when out_host != nullptr, copied to the host (synchronising the stream).
int vec_dots(sg_ctx* h, const double* V, size_t ldv, int nv, const double* w, size_t N, bool with_ww, double* out_host) {
  int rc = ensure_reduction(h);
  if (rc) return rc;
  if (nv < 0 || nv > 32) return sg_fail(h, SG_E_ARG, "dots: at most 32 vectors per call");
  const int g = red_grid(h, N);
  double* out = h->red_out;
  if (nv <= 4) k_dots<4><<<g, NT, 0, h->stream>>>(V, ldv, nv, w, N, with_ww, h->red_partial, out, h->red_count);
  else if (nv <= 8) k_dots<8><<<g, NT, 0, h->stream>>>(V, ldv, nv, w, N, with_ww, h->red_partial, out, h->red_count);
  else if (nv <= 16) k_dots<16><<<g, NT, 0, h->stream>>>(V, ldv, nv, w, N, with_ww, h->red_partial, out, h->red_count);
  else k_dots<32><<<g, NT, 0, h->stream>>>(V, ldv, nv, w, N, with_ww, h->red_partial, out, h->red_count);
  SG_CUDA(h, cudaGetLastError());
  count_launch(h);
  if (out_host) {
    SG_CUDA(h, cudaMemcpyAsync(h->red_host, out, sizeof(double) * (nv + 1), cudaMemcpyDeviceToHost, h->stream));
    SG_CUDA(h, cudaStreamSynchronize(h->stream));
    std::copy(h->red_host, h->red_host + nv + (with_ww ? 1 : 0), out_host);
  }
  return SG_OK;
}

// w -= V hc (hc on the device), ||w||^2 -> *nrm2_host (synchronises when nrm2_host != nullptr)
int vec_axpys_norm(sg_ctx* h, const double* V, size_t ldv, int nv, const double* hc, double* w, size_t N, double* nrm2_host) {
  int rc = ensure_reduction(h);
  if (rc) return rc;
  if (nv < 0 || nv > 32) return sg_fail(h, SG_E_ARG, "axpys: at most 32 vectors per call");
  const int g = red_grid(h, N);
  double* out = h->red_out + MAXOUT;
  unsigned* cnt = h->red_count + 1;
  if (nv <= 4) k_axpys<4><<<g, NT, 0, h->stream>>>(V, ldv, nv, hc, w, N, h->red_partial, out, cnt);
  else if (nv <= 8) k_axpys<8><<<g, NT, 0, h->stream>>>(V, ldv, nv, hc, w, N, h->red_partial, out, cnt);
  else if (nv <= 16) k_axpys<16><<<g, NT, 0, h->stream>>>(V, ldv, nv, hc, w, N, h->red_partial, out, cnt);
  else k_axpys<32><<<g, NT, 0, h->stream>>>(V, ldv, nv, hc, w, N, h->red_partial, out, cnt);
  SG_CUDA(h, cudaGetLastError());
  count_launch(h);
  if (nrm2_host) {
    SG_CUDA(h, cudaMemcpyAsync(h->red_host + MAXOUT, out, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    SG_CUDA(h, cudaStreamSynchronize(h->stream));
    *nrm2_host = h->red_host[MAXOUT];
  }
  return SG_OK;
}

// copy count results of reduction slot (0 dots, 1 axpys norm, 3 dot pairs) to the host
int copy_red(sg_ctx* h, int slot, int count, double* out_host) {
  SG_CUDA(h, cudaMemcpyAsync(h->red_host + slot * MAXOUT, h->red_out + slot * MAXOUT, sizeof(double) * count,
                             cudaMemcpyDeviceToHost, h->stream));
  SG_CUDA(h, cudaStreamSynchronize(h->stream));
  std::copy(h->red_host + slot * MAXOUT, h->red_host + slot * MAXOUT + count, out_host);
  return SG_OK;
}

int vec_scale(sg_ctx* h, const double* w, double* v, size_t N, double s) {
  k_scale<<<grid_for(N), 256, 0, h->stream>>>(w, v, N, s);
  SG_CUDA(h, cudaGetLastError());
  count_launch(h);
  return SG_OK;
}

int vec_update(sg_ctx* h, double* U, int zprec, const void* Z, size_t ldz, int nz, const double* y_host, size_t N) {
  int rc = ensure_reduction(h);
  if (rc) return rc;
  const size_t es = prec_size(zprec);
  for (int c0 = 0; c0 < nz; c0 += 16) {
    const int cn = std::min(16, nz - c0);
    double* ydev = h->red_out + 2 * MAXOUT;
    std::copy(y_host + c0, y_host + c0 + cn, h->red_host + 2 * MAXOUT);
    SG_CUDA(h, cudaMemcpyAsync(ydev, h->red_host + 2 * MAXOUT, sizeof(double) * cn, cudaMemcpyHostToDevice, h->stream));
    const void* Zc = (const char*)Z + es * (size_t)c0 * ldz;
    if (zprec == SG_F64) k_update<double, 16><<<grid_for(N), 256, 0, h->stream>>>(U, (const double*)Zc, ldz, cn, ydev, N);
    else if (zprec == SG_F32) k_update<float, 16><<<grid_for(N), 256, 0, h->stream>>>(U, (const float*)Zc, ldz, cn, ydev, N);
    else k_update<bf16, 16><<<grid_for(N), 256, 0, h->stream>>>(U, (const bf16*)Zc, ldz, cn, ydev, N);
    SG_CUDA(h, cudaGetLastError());
    count_launch(h);
    // the host staging slot is reused by the next chunk: wait for this copy
    SG_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  return SG_OK;
}

int vec_cast(sg_ctx* h, int iprec, const void* in, int oprec, void* out, size_t N) {
  const int g = grid_for(N);
#define SG_C(TI, TO) k_cast<TI, TO><<<g, 256, 0, h->stream>>>((const TI*)in, (TO*)out, N)
  if (iprec == SG_F64 && oprec == SG_F32) SG_C(double, float);
  else if (iprec == SG_F64 && oprec == SG_BF16) SG_C(double, bf16);
  else if (iprec == SG_F32 && oprec == SG_F64) SG_C(float, double);
  else if (iprec == SG_BF16 && oprec == SG_F64) SG_C(bf16, double);
  else if (iprec == oprec) {
    SG_CUDA(h, cudaMemcpyAsync(out, in, N * prec_size(iprec), cudaMemcpyDeviceToDevice, h->stream));
  } else return sg_fail(h, SG_E_ARG, "cast: unsupported precision pair");
#undef SG_C
  SG_CUDA(h, cudaGetLastError());
  count_launch(h);
  return SG_OK;
}

int vec_axpby(sg_ctx* h, double a, const double* x, double b, double* y, size_t N) {
  k_axpby<<<grid_for(N), 256, 0, h->stream>>>(a, x, b, y, N);
  SG_CUDA(h, cudaGetLastError());
  count_launch(h);
  return SG_OK;
}

int vec_axpy_prec(sg_ctx* h, double a, int xprec, const void* x, double* y, size_t N) {
  if (xprec == SG_F64) k_axpy_prec<double><<<grid_for(N), 256, 0, h->stream>>>(a, (const double*)x, y, N);
  else if (xprec == SG_F32) k_axpy_prec<float><<<grid_for(N), 256, 0, h->stream>>>(a, (const float*)x, y, N);
  else k_axpy_prec<bf16><<<grid_for(N), 256, 0, h->stream>>>(a, (const bf16*)x, y, N);
  SG_CUDA(h, cudaGetLastError());
  count_launch(h);
  return SG_OK;
}

int vec_dot_pairs(sg_ctx* h, int npairs, const double* const* xs, const void* const* ys, const int* yprecs, size_t N,
                  double* out_host) {
  int rc = ensure_reduction(h);
  if (rc) return rc;
  if (npairs < 1 || npairs > 4) return sg_fail(h, SG_E_ARG, "dot pairs: 1..4");
  DotPairs D{};
  D.n = npairs;
  for (int q = 0; q < npairs; ++q) { D.x[q] = xs[q]; D.y[q] = ys[q]; D.yp[q] = yprecs[q]; }
  double* out = h->red_out + 3 * MAXOUT;
  k_dotpairs<<<red_grid(h, N), NT, 0, h->stream>>>(D, N, h->red_partial, out, h->red_count + 2);
  SG_CUDA(h, cudaGetLastError());
  count_launch(h);
  SG_CUDA(h, cudaMemcpyAsync(h->red_host + 3 * MAXOUT, out, sizeof(double) * npairs, cudaMemcpyDeviceToHost, h->stream));
  SG_CUDA(h, cudaStreamSynchronize(h->stream));
  std::copy(h->red_host + 3 * MAXOUT, h->red_host + 3 * MAXOUT + npairs, out_host);
  return SG_OK;
}

int adj_cell_forms(sg_ctx* h, const double* U, const double* L, double* g_abar) {
  k_cell_forms<<<grid_for(h->Nc), 256, 0, h->stream>>>(U, L, g_abar, h->n, h->m, h->P, h->Nx);
  SG_CUDA(h, cudaGetLastError());
  count_launch(h);
  return SG_OK;
}

int objective_dots(sg_ctx* h, const double* U, double* mu_host) {
  int rc = ensure_reduction(h);
  if (rc) return rc;
  const double hh = 1.0 / (h->n - 1);
  double* mu = h->pvec;
  k_row_sums<<<h->P, NT, 0, h->stream>>>(U, h->Nx, hh * hh, mu);
  SG_CUDA(h, cudaGetLastError());
  count_launch(h);
  SG_CUDA(h, cudaMemcpyAsync(mu_host, mu, sizeof(double) * h->P, cudaMemcpyDeviceToHost, h->stream));
  SG_CUDA(h, cudaStreamSynchronize(h->stream));
  return SG_OK;
}

int objective_grad(sg_ctx* h, const double* mu_dev, double* G) {
  const double hh = 1.0 / (h->n - 1);
  k_obj_grad<<<grid_for(h->Nx * h->P), 256, 0, h->stream>>>(mu_dev, G, h->Nx, h->P, hh * hh);
  SG_CUDA(h, cudaGetLastError());
  count_launch(h);
  return SG_OK;
}
