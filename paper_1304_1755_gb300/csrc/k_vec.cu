// FP64 Krylov vector kernels: fused multi-dot (Arnoldi h = V^T w), fused
// multi-axpy with norm (w -= V h, ||w||^2), scaling, solution updates, casts and
// the small fused updates of GPCG[1] / PCG (Sec. 4.2).  Reductions are
// deterministic: warp shuffles, a per-block partial in global memory and a
// fixed-order sum by the last block to finish.
#include <algorithm>
#include <vector>

#include "df64.cuh"
#include "sg_internal.h"
#include "update_q.cuh"

#define SG_NV_CASES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16) \
  X(17) X(18) X(19) X(20) X(21) X(22) X(23) X(24) X(25) X(26) X(27) X(28) X(29) X(30) X(31) X(32)

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
    // final sum over the block partials: each warp owns outputs o = warp, warp + 8, ...; its lanes
    // stride over the blocks in a fixed order and the warp reduces with shuffles (deterministic)
    __threadfence();
    for (int o = warp; o < nout; o += NT / 32) {
      double v = 0;
      for (int b = lane; b < (int)gridDim.x; b += 32) v += __ldcg(partial + (size_t)b * MAXOUT + o);
      for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
      if (lane == 0) out[o] = v;
    }
    if (threadIdx.x == 0) *counter = 0u;
  }
}

// h_l = <V_l, w> for l < NV (exact count: no predicated slots) and, in slot NV, <w, w>.
template <int NV>
__global__ void __launch_bounds__(NT) k_dots(const double* __restrict__ V, size_t ldv, const double* __restrict__ w,
                                             size_t N, int with_ww, double* partial, double* out, unsigned* counter) {
  // N: padded length (even; the padding holds zeros); 16-byte loads of two elements
  double acc[NV + 1];
#pragma unroll
  for (int l = 0; l <= NV; ++l) acc[l] = 0;
  const size_t n2 = N / 2;
  for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n2; q += (size_t)gridDim.x * NT) {
    const double2 wv = ((const double2*)w)[q];
#pragma unroll
    for (int l = 0; l < NV; ++l) {
      const double2 v = ((const double2*)(V + (size_t)l * ldv))[q];
      acc[l] = fma(v.x, wv.x, fma(v.y, wv.y, acc[l]));
    }
    if (with_ww) acc[NV] = fma(wv.x, wv.x, fma(wv.y, wv.y, acc[NV]));
  }
  reduce_out<NV + 1>(acc, partial, out, counter, NV + (with_ww ? 1 : 0));
}

// w -= sum_l hc_l V_l and ||w||^2
template <int NV>
__global__ void __launch_bounds__(NT) k_axpys(const double* __restrict__ V, size_t ldv, const double* __restrict__ hc,
                                              double* __restrict__ w, size_t N, double* partial, double* out,
                                              unsigned* counter) {
  double c[NV];
#pragma unroll
  for (int l = 0; l < NV; ++l) c[l] = hc[l];
  double acc[1] = {0};
  const size_t n2 = N / 2;
  for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n2; q += (size_t)gridDim.x * NT) {
    double2 v = ((double2*)w)[q];
#pragma unroll
    for (int l = 0; l < NV; ++l) {
      const double2 x = ((const double2*)(V + (size_t)l * ldv))[q];
      v.x = fma(-c[l], x.x, v.x);
      v.y = fma(-c[l], x.y, v.y);
    }
    ((double2*)w)[q] = v;
    acc[0] = fma(v.x, v.x, fma(v.y, v.y, acc[0]));
  }
  reduce_out<1>(acc, partial, out, counter, 1);
}

// ---- double-float vectors: hi[0..N), lo[N..2N) ------------------------------
__device__ __forceinline__ double dacc_to_double(dacc a) { return (double)a.s + (double)a.c; }

template <int NV>
__global__ void __launch_bounds__(NT) k_dots_df(const float* __restrict__ V, size_t ldv, const float* __restrict__ w,
                                                size_t N, int with_ww, double* partial, double* out,
                                                unsigned* counter) {
  // N: padded length (multiple of 4, lo array at +N, padding zero); 16-byte loads of 4 elements
  dacc acc[NV + 1];
#pragma unroll
  for (int l = 0; l <= NV; ++l) acc[l] = dacc_zero();
  const size_t n4 = N / 4;
  for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n4; q += (size_t)gridDim.x * NT) {
    const float4 wh = ((const float4*)w)[q], wl = ((const float4*)(w + N))[q];
#pragma unroll
    for (int l = 0; l < NV; ++l) {
      const float4 vh = ((const float4*)(V + (size_t)l * ldv))[q];
      const float4 vl = ((const float4*)(V + (size_t)l * ldv + N))[q];
      dacc_fma(acc[l], df2{vh.x, vl.x}, df2{wh.x, wl.x});
      dacc_fma(acc[l], df2{vh.y, vl.y}, df2{wh.y, wl.y});
      dacc_fma(acc[l], df2{vh.z, vl.z}, df2{wh.z, wl.z});
      dacc_fma(acc[l], df2{vh.w, vl.w}, df2{wh.w, wl.w});
    }
    if (with_ww) {
      dacc_fma(acc[NV], df2{wh.x, wl.x}, df2{wh.x, wl.x});
      dacc_fma(acc[NV], df2{wh.y, wl.y}, df2{wh.y, wl.y});
      dacc_fma(acc[NV], df2{wh.z, wl.z}, df2{wh.z, wl.z});
      dacc_fma(acc[NV], df2{wh.w, wl.w}, df2{wh.w, wl.w});
    }
  }
  double r[NV + 1];
#pragma unroll
  for (int l = 0; l <= NV; ++l) r[l] = dacc_to_double(acc[l]);
  reduce_out<NV + 1>(r, partial, out, counter, NV + (with_ww ? 1 : 0));
}

template <int NV>
__global__ void __launch_bounds__(NT) k_axpys_df(const float* __restrict__ V, size_t ldv, const double* __restrict__ hc,
                                                 float* __restrict__ w, size_t N, double* partial, double* out,
                                                 unsigned* counter) {
  df2 c[NV];
#pragma unroll
  for (int l = 0; l < NV; ++l) c[l] = df_from_double(-hc[l]);
  dacc nn = dacc_zero();
  const size_t n4 = N / 4;
  for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n4; q += (size_t)gridDim.x * NT) {
    const float4 wh = ((const float4*)w)[q], wl = ((const float4*)(w + N))[q];
    dacc v0 = {wh.x, wl.x}, v1 = {wh.y, wl.y}, v2 = {wh.z, wl.z}, v3 = {wh.w, wl.w};
#pragma unroll
    for (int l = 0; l < NV; ++l) {
      const float4 xh = ((const float4*)(V + (size_t)l * ldv))[q];
      const float4 xl = ((const float4*)(V + (size_t)l * ldv + N))[q];
      dacc_fma(v0, c[l], df2{xh.x, xl.x});
      dacc_fma(v1, c[l], df2{xh.y, xl.y});
      dacc_fma(v2, c[l], df2{xh.z, xl.z});
      dacc_fma(v3, c[l], df2{xh.w, xl.w});
    }
    const df2 r0 = dacc_get(v0), r1 = dacc_get(v1), r2 = dacc_get(v2), r3 = dacc_get(v3);
    ((float4*)w)[q] = make_float4(r0.hi, r1.hi, r2.hi, r3.hi);
    ((float4*)(w + N))[q] = make_float4(r0.lo, r1.lo, r2.lo, r3.lo);
    dacc_fma(nn, r0, r0);
    dacc_fma(nn, r1, r1);
    dacc_fma(nn, r2, r2);
    dacc_fma(nn, r3, r3);
  }
  double acc[1] = {dacc_to_double(nn)};
  reduce_out<1>(acc, partial, out, counter, 1);
}

// U += sum_l y_l Z_l for a double-float U (hi at U, lo at U + lo) and nz FP32/BF16 vectors at
// stride ldz; four elements per thread with 16-byte (8-byte for BF16) loads.  ldz and lo are
// multiples of 4 and the arrays 16-byte aligned; elements at and beyond N are left unchanged.
template <typename TZ> struct Z4;
template <> struct Z4<float> {
  static __device__ __forceinline__ float4 ld(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
};
template <> struct Z4<bf16> {
  static __device__ __forceinline__ float4 ld(const bf16* p) {
    const uint2 r = __ldg(reinterpret_cast<const uint2*>(p));
    return make_float4(__uint_as_float(r.x << 16), __uint_as_float(r.x & 0xffff0000u), __uint_as_float(r.y << 16),
                       __uint_as_float(r.y & 0xffff0000u));
  }
};

template <typename TZ>
__global__ void k_update_df(float* __restrict__ U, const TZ* __restrict__ Z, size_t ldz, int nz,
                            const double* __restrict__ y, size_t N, size_t lo) {
  __shared__ df2 cs[SG_MAX_RESTART];
  for (int l = threadIdx.x; l < nz; l += blockDim.x) cs[l] = df_from_double(y[l]);
  __syncthreads();
  const size_t n4 = (N + 3) / 4;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n4; q += (size_t)gridDim.x * blockDim.x) {
    const size_t i = 4 * q;
    const float4 uh = reinterpret_cast<const float4*>(U)[q], ul = reinterpret_cast<const float4*>(U + lo)[q];
    dacc u0 = {uh.x, ul.x}, u1 = {uh.y, ul.y}, u2 = {uh.z, ul.z}, u3 = {uh.w, ul.w};
#pragma unroll 4
    for (int l = 0; l < nz; ++l) {
      const float4 z = Z4<TZ>::ld(Z + (size_t)l * ldz + i);
      const df2 c = cs[l];
      dacc_fma(u0, c, z.x);
      dacc_fma(u1, c, z.y);
      dacc_fma(u2, c, z.z);
      dacc_fma(u3, c, z.w);
    }
    df2 r0 = dacc_get(u0), r1 = dacc_get(u1), r2 = dacc_get(u2), r3 = dacc_get(u3);
    if (i + 1 >= N) r1 = {uh.y, ul.y};
    if (i + 2 >= N) r2 = {uh.z, ul.z};
    if (i + 3 >= N) r3 = {uh.w, ul.w};
    reinterpret_cast<float4*>(U)[q] = make_float4(r0.hi, r1.hi, r2.hi, r3.hi);
    reinterpret_cast<float4*>(U + lo)[q] = make_float4(r0.lo, r1.lo, r2.lo, r3.lo);
  }
}

__global__ void k_fill(double* __restrict__ y, size_t N, double v) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) y[i] = v;
}

// F = e_0 (x) (w f): the mean PC block w f_s (w when f is null), every other block zero
__global__ void k_load(const double* __restrict__ f, double w, double* __restrict__ F, size_t Nx, size_t N) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    F[i] = i < Nx ? (f ? w * f[i] : w) : 0.0;
}

// split an FP64 vector into a double-float vector; positions [N, lo) of both halves are zeroed
// (the padding of Krylov vectors must stay zero)
__global__ void k_df_from_f64(const double* __restrict__ x, float* __restrict__ y, size_t N, size_t lo) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < lo; i += (size_t)gridDim.x * blockDim.x) {
    const df2 r = i < N ? df_from_double(x[i]) : df2{0.f, 0.f};
    y[i] = r.hi;
    y[i + lo] = r.lo;
  }
}

__global__ void k_df_to_f64(const float* __restrict__ x, double* __restrict__ y, size_t N, size_t lo) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (double)x[i] + (double)x[i + lo];
}

template <typename TZ, int NV>
__global__ void k_update(double* __restrict__ U, const TZ* __restrict__ Z, size_t ldz, int nz,
                         const double* __restrict__ y, size_t N) {
  if constexpr (sizeof(TZ) == 8) {
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
  } else {
    // FP32 / BF16 z: the sum over l in double-float (FP32 instructions), added to U in FP64 once.  The
    // coefficients as double-float sit in shared memory (zero past nz), formed once per CTA; every
    // column load is issued before the sums (slots past nz re-read the last column).
    __shared__ float2 kc[NV];
    for (int l = threadIdx.x; l < NV; l += blockDim.x) {
      const df2 c = df_from_double(l < nz ? y[l] : 0.0);
      kc[l] = make_float2(c.hi, c.lo);
    }
    __syncthreads();
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
      float zv[NV];
#pragma unroll
      for (int l = 0; l < NV; ++l) zv[l] = ld_as<float>(Z + (size_t)min(l, nz - 1) * ldz + i);
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
  h->red_blocks = 152 * 8;
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
  (void)0;
  switch (nv) {
    case 0: k_dots<0><<<g, NT, 0, h->stream>>>(V, ldv, w, N, with_ww, h->red_partial, out, h->red_count); break;
#define SG_C(K) \
    case K: k_dots<K><<<g, NT, 0, h->stream>>>(V, ldv, w, N, with_ww, h->red_partial, out, h->red_count); break;
    SG_NV_CASES(SG_C)
#undef SG_C
  }
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
  if (nv < 1 || nv > 32) return sg_fail(h, SG_E_ARG, "axpys: 1..32 vectors per call");
  const int g = red_grid(h, N);
  double* out = h->red_out + MAXOUT;
  unsigned* cnt = h->red_count + 1;
  switch (nv) {
#define SG_C(K) \
    case K: k_axpys<K><<<g, NT, 0, h->stream>>>(V, ldv, hc, w, N, h->red_partial, out, cnt); break;
    SG_NV_CASES(SG_C)
#undef SG_C
  }
  SG_CUDA(h, cudaGetLastError());
  count_launch(h);
  if (nrm2_host) {
    SG_CUDA(h, cudaMemcpyAsync(h->red_host + MAXOUT, out, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    SG_CUDA(h, cudaStreamSynchronize(h->stream));
    *nrm2_host = h->red_host[MAXOUT];
  }
  return SG_OK;
}

// double-float versions: V_l hi at V + l*ldv (lo at + N); results in reduction slots 0 / 1
int df_dots(sg_ctx* h, const float* V, size_t ldv, int nv, const float* w, size_t N, bool with_ww) {
  int rc = ensure_reduction(h);
  if (rc) return rc;
  if (nv < 0 || nv > 32) return sg_fail(h, SG_E_ARG, "dots: at most 32 vectors per call");
  const int g = red_grid(h, N);
  double* out = h->red_out;
  switch (nv) {
    case 0: k_dots_df<0><<<g, NT, 0, h->stream>>>(V, ldv, w, N, with_ww, h->red_partial, out, h->red_count); break;
#define SG_C(K) \
    case K: k_dots_df<K><<<g, NT, 0, h->stream>>>(V, ldv, w, N, with_ww, h->red_partial, out, h->red_count); break;
    SG_NV_CASES(SG_C)
#undef SG_C
  }
  SG_CUDA(h, cudaGetLastError());
  count_launch(h);
  return SG_OK;
}

int df_axpys_norm(sg_ctx* h, const float* V, size_t ldv, int nv, const double* hc, float* w, size_t N) {
  int rc = ensure_reduction(h);
  if (rc) return rc;
  if (nv < 1 || nv > 32) return sg_fail(h, SG_E_ARG, "axpys: 1..32 vectors per call");
  const int g = red_grid(h, N);
  double* out = h->red_out + MAXOUT;
  unsigned* cnt = h->red_count + 1;
  switch (nv) {
#define SG_C(K) \
    case K: k_axpys_df<K><<<g, NT, 0, h->stream>>>(V, ldv, hc, w, N, h->red_partial, out, cnt); break;
    SG_NV_CASES(SG_C)
#undef SG_C
  }
  SG_CUDA(h, cudaGetLastError());
  count_launch(h);
  return SG_OK;
}

int df_update(sg_ctx* h, float* U, size_t lo, int zprec, const void* Z, size_t ldz, int nz, const double* y_host,
              size_t N) {
  int rc = ensure_reduction(h);
  if (rc) return rc;
  if (nz <= 0) return SG_OK;
  if (nz > MAXOUT || ldz % 4 || lo % 4) return sg_fail(h, SG_E_ARG, "df update: bad layout");
  double* ydev = h->red_out + 2 * MAXOUT;
  std::copy(y_host, y_host + nz, h->red_host + 2 * MAXOUT);
  SG_CUDA(h, cudaMemcpyAsync(ydev, h->red_host + 2 * MAXOUT, sizeof(double) * nz, cudaMemcpyHostToDevice, h->stream));
  const int g = grid_for((N + 3) / 4);
  if (zprec == SG_F32) k_update_df<float><<<g, 256, 0, h->stream>>>(U, (const float*)Z, ldz, nz, ydev, N, lo);
  else if (zprec == SG_BF16) k_update_df<bf16><<<g, 256, 0, h->stream>>>(U, (const bf16*)Z, ldz, nz, ydev, N, lo);
  else return sg_fail(h, SG_E_ARG, "df update: Z must be FP32 or BF16");
  SG_CUDA(h, cudaGetLastError());
  count_launch(h);
  // the host staging slot is reused by the next call: wait for this copy
  SG_CUDA(h, cudaStreamSynchronize(h->stream));
  return SG_OK;
}

int vec_fill(sg_ctx* h, double* y, size_t N, double v) {
  k_fill<<<grid_for(N), 256, 0, h->stream>>>(y, N, v);
  SG_CUDA(h, cudaGetLastError());
  count_launch(h);
  return SG_OK;
}

// per-block max |z| as float bits (non-negative floats order like their bit patterns)
__global__ void k_block_absmax(const float* __restrict__ Z, size_t Nx, unsigned* __restrict__ qmax) {
  const float* z = Z + (size_t)blockIdx.y * Nx;
  unsigned m = 0;
  const size_t st = (size_t)gridDim.x * blockDim.x;
  size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  for (; s + 3 * st < Nx; s += 4 * st) {                      // four independent loads in flight
    const float a = __ldg(z + s), b = __ldg(z + s + st), c = __ldg(z + s + 2 * st), d = __ldg(z + s + 3 * st);
    m = max(max(m, __float_as_uint(fabsf(a))), max(__float_as_uint(fabsf(b)),
                                                    max(__float_as_uint(fabsf(c)), __float_as_uint(fabsf(d)))));
  }
  for (; s < Nx; s += st) m = max(m, __float_as_uint(fabsf(z[s])));
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(qmax + blockIdx.y, m);
}

int block_absmax(sg_ctx* h, const float* Z, unsigned* qmax) {
  SG_CUDA(h, cudaMemsetAsync(qmax, 0, sizeof(unsigned) * h->P, h->stream));
  // about eight warps per SM per block row of the grid, each thread with 16 or more values
  const int gx = (int)std::max<size_t>(1, std::min<size_t>((h->Nx + 4095) / 4096, (size_t)(152 * 8 + h->P - 1) / h->P));
  k_block_absmax<<<dim3(gx, h->P), 256, 0, h->stream>>>(Z, h->Nx, qmax);
  SG_CUDA(h, cudaGetLastError());
  count_launch(h);
  return SG_OK;
}


// FP64 U += sum_l y_l z'_l over NV grid-read FP32 columns (update_q_block); grid x over the nodes of a
// block, grid y over the blocks; the per-column constants are formed once per CTA in shared memory.
template <int NV>
__global__ void k_update_q(double* __restrict__ U, const float* __restrict__ Z, size_t ldz,
                           const double* __restrict__ y, size_t Nx, const unsigned* __restrict__ qmax, int P) {
  const int b = blockIdx.y;
  __shared__ float4 kc[NV];
  for (int l = threadIdx.x; l < NV; l += blockDim.x) {
    const df2 c = df_from_double(y[l]);
    const unsigned mb = qmax[(size_t)l * P + b];
    kc[l] = make_float4(c.hi, c.lo, qgrid_scale(mb), qgrid_quantum(mb));
  }
  __syncthreads();
  update_q_block<NV>(U, Z, ldz, kc, NV, Nx, b);
}

// double-float U (hi at U, lo at U + lo) += sum_l y_l z'_l
__global__ void k_update_df_q(float* __restrict__ U, size_t lo, const float* __restrict__ Z, size_t ldz, int nz,
                              const double* __restrict__ y, size_t Nx, const unsigned* __restrict__ qmax, int P) {
  __shared__ df2 cs[SG_MAX_RESTART];
  __shared__ float sc[SG_MAX_RESTART], qu[SG_MAX_RESTART];
  const int b = blockIdx.y;
  for (int l = threadIdx.x; l < nz; l += blockDim.x) {
    cs[l] = df_from_double(y[l]);
    const unsigned mb = qmax[(size_t)l * P + b];
    sc[l] = qgrid_scale(mb), qu[l] = qgrid_quantum(mb);
  }
  __syncthreads();
  float* Uh = U + (size_t)b * Nx;
  float* Ul = Uh + lo;
  const float* Zb = Z + (size_t)b * Nx;
  for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < Nx; s += (size_t)gridDim.x * blockDim.x) {
    dacc u = {Uh[s], Ul[s]};
#pragma unroll 4
    for (int l = 0; l < nz; ++l) dacc_fma(u, cs[l], qgrid_value(Zb[(size_t)l * ldz + s], sc[l], qu[l]));
    const df2 r = dacc_get(u);
    Uh[s] = r.hi, Ul[s] = r.lo;
  }
}

int vec_update_q(sg_ctx* h, double* U, const float* Z, size_t ldz, int nz, const double* y_host, size_t N,
                 const unsigned* qmax) {
  int rc = ensure_reduction(h);
  if (rc) return rc;
  if (N != h->Nx * (size_t)h->P) return sg_fail(h, SG_E_ARG, "grid update: bad length");
  const int gx = (int)std::max<size_t>(1, std::min<size_t>((h->Nx + 4095) / 4096, 64));
  for (int c0 = 0; c0 < nz; c0 += 16) {
    const int cn = std::min(16, nz - c0);
    double* ydev = h->red_out + 2 * MAXOUT;
    std::copy(y_host + c0, y_host + c0 + cn, h->red_host + 2 * MAXOUT);
    SG_CUDA(h, cudaMemcpyAsync(ydev, h->red_host + 2 * MAXOUT, sizeof(double) * cn, cudaMemcpyHostToDevice, h->stream));
    const float* Zc = Z + (size_t)c0 * ldz;
    const unsigned* qc = qmax + (size_t)c0 * h->P;
    switch (cn) {                                  // the exact column count: no idle slots
#define SG_C(K) \
      case K: k_update_q<K><<<dim3(gx, h->P), 256, 0, h->stream>>>(U, Zc, ldz, ydev, h->Nx, qc, h->P); break;
      SG_C(1) SG_C(2) SG_C(3) SG_C(4) SG_C(5) SG_C(6) SG_C(7) SG_C(8) SG_C(9) SG_C(10) SG_C(11) SG_C(12) SG_C(13)
      SG_C(14) SG_C(15) SG_C(16)
#undef SG_C
    }
    SG_CUDA(h, cudaGetLastError());
    count_launch(h);
    SG_CUDA(h, cudaStreamSynchronize(h->stream));      // the host staging slot is reused by the next chunk
  }
  return SG_OK;
}

int df_update_q(sg_ctx* h, float* U, size_t lo, const float* Z, size_t ldz, int nz, const double* y_host, size_t N,
                const unsigned* qmax) {
  int rc = ensure_reduction(h);
  if (rc) return rc;
  if (nz <= 0) return SG_OK;
  if (nz > MAXOUT || N != h->Nx * (size_t)h->P) return sg_fail(h, SG_E_ARG, "grid df update: bad layout");
  double* ydev = h->red_out + 2 * MAXOUT;
  std::copy(y_host, y_host + nz, h->red_host + 2 * MAXOUT);
  SG_CUDA(h, cudaMemcpyAsync(ydev, h->red_host + 2 * MAXOUT, sizeof(double) * nz, cudaMemcpyHostToDevice, h->stream));
  const int gx = (int)std::max<size_t>(1, std::min<size_t>((h->Nx + 4095) / 4096, 64));
  k_update_df_q<<<dim3(gx, h->P), 256, 0, h->stream>>>(U, lo, Z, ldz, nz, ydev, h->Nx, qmax, h->P);
  SG_CUDA(h, cudaGetLastError());
  count_launch(h);
  SG_CUDA(h, cudaStreamSynchronize(h->stream));
  return SG_OK;
}

int vec_load(sg_ctx* h, const double* f, double w, double* F) {
  const size_t N = h->Nx * (size_t)h->P;
  k_load<<<grid_for(N), 256, 0, h->stream>>>(f, w, F, h->Nx, N);
  SG_CUDA(h, cudaGetLastError());
  count_launch(h);
  return SG_OK;
}

int df_from_f64(sg_ctx* h, const double* x, float* y, size_t N, size_t lo) {
  k_df_from_f64<<<grid_for(N), 256, 0, h->stream>>>(x, y, N, lo);
  SG_CUDA(h, cudaGetLastError());
  count_launch(h);
  return SG_OK;
}

int df_to_f64(sg_ctx* h, const float* x, double* y, size_t N, size_t lo) {
  k_df_to_f64<<<grid_for(N), 256, 0, h->stream>>>(x, y, N, lo);
  SG_CUDA(h, cudaGetLastError());
  count_launch(h);
  return SG_OK;
}

// copy count results of reduction slot (0 dots, 1 axpys norm, 3 dot pairs) to the host
int upload_red(sg_ctx* h, int slot, const double* host, int count) {
  if (count > MAXOUT) return sg_fail(h, SG_E_ARG, "reduction slot overflow");
  std::copy(host, host + count, h->red_host + slot * MAXOUT);
  SG_CUDA(h, cudaMemcpyAsync(h->red_out + slot * MAXOUT, h->red_host + slot * MAXOUT, sizeof(double) * count,
                             cudaMemcpyHostToDevice, h->stream));
  return SG_OK;
}

const double* red_slot(const sg_ctx* h, int slot) { return h->red_out + slot * MAXOUT; }

int copy_red(sg_ctx* h, int slot, int count, double* out_host) {
  SG_CUDA(h, cudaMemcpyAsync(h->red_host + slot * MAXOUT, h->red_out + slot * MAXOUT, sizeof(double) * count,
                             cudaMemcpyDeviceToHost, h->stream));
  SG_CUDA(h, cudaStreamSynchronize(h->stream));
  std::copy(h->red_host + slot * MAXOUT, h->red_host + slot * MAXOUT + count, out_host);
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
