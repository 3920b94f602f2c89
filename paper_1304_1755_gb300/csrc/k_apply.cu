// K1: matrix-free SG operator  Y_i = sum_k sum_j G_k(i,j) K_k X_j  (Eq. tensor-product),
// and its restriction to the lower / upper degree couplings (the stage update of the
// block-triangular sweep, Sec. 4.2).
//
// K_k X_j = sum_e c_k(e) K_ref^(e) X_j with K_ref the Q1 element matrix of the
// Laplacian on a square cell, corners SW(a) SE(b) NE(c) NW(d):
//   K_ref = (1/6)[4 -1 -2 -1; -1 4 -1 -2; -2 -1 4 -1; -1 -2 -1 4]
//         = (1/2) f1 f1^T + (1/2) f2 f2^T + (1/6) f3 f3^T,
//   f1 = (1,0,-1,0), f2 = (0,1,0,-1), f3 = (1,-1,1,-1).
// For output row i and cell e the kernel first mixes the coupled columns at the
// cell's four corners,  t(v) = sum_t c_{k_t}(e) G_{k_t}(i, j_t) X_{j_t}(v),  then
// applies K_ref through the three features d1 = ta - tc, d2 = tb - td,
// hg = ta - tb + tc - td and scatters  A = d1/2, B = d2/2, C = hg/6  to the corners:
// a += A + C, b += B - C, c += C - A, d += -B - C.
//
// One thread per cell: a CTA owns 32 x 8 cells and produces the 31 x 7 nodes
// whose four cells it holds (cell results meet in shared memory), looping over
// ROWS output rows.  The 1-D grid enumerates (tile, row group) with row groups
// fastest, so a tile's input columns are reused from L2 by neighbouring CTAs.
//
// Arithmetic policies: FP32, FP64 (IEEE double) and DF (double-float, see df64.cuh;
// used where FP64-class accuracy is needed at FP32 throughput).
#include <type_traits>

#include "df64.cuh"
#include "sg_internal.h"

namespace {
constexpr int CXN = 32, CYN = 8, NT = CXN * CYN;   // cells per CTA
constexpr int OXN = CXN - 1, OYN = CYN - 1;        // output nodes per CTA
constexpr int ROWS = 4;
constexpr int MAXT = 16;                            // staged coupling terms per row (more: read from global)

struct ApplyArgs {
  const void* X;
  size_t xlo;          // offset of the lo array for double-float storage
  void* Y;
  size_t ylo;
  const void* R;
  size_t rlo;
  const double* c64;
  const float* c32;
  const df2* cdf;
  const df2* wdf;      // optional table of weights c_k(e) gamma_n as double-float, slot-major
  const int* ws;       // weight slot of each term
  const int* row_ptr;
  const int* tj;
  const int* tk;
  const double* g64;
  const float* g32;
  const df2* gdf;
  int row0, nrows, ybase, rbase, n, m;
  size_t Nx, Nc;
  int tiles_x, ngroups;
};

// ---- storage access --------------------------------------------------------
struct DFS {};   // tag: double-float storage, hi array at p, lo array at p + lo

template <typename TS> struct Load;
template <> struct Load<double> {
  typedef double Z;
  static __device__ __forceinline__ Z at(const void* p, size_t, size_t i) { return ((const double*)p)[i]; }
  static __device__ __forceinline__ Z zero() { return 0.0; }
};
template <> struct Load<float> {
  typedef float Z;
  static __device__ __forceinline__ Z at(const void* p, size_t, size_t i) { return ((const float*)p)[i]; }
  static __device__ __forceinline__ Z zero() { return 0.f; }
};
template <> struct Load<bf16> {
  typedef float Z;
  static __device__ __forceinline__ Z at(const void* p, size_t, size_t i) { return __bfloat162float(((const bf16*)p)[i]); }
  static __device__ __forceinline__ Z zero() { return 0.f; }
};
template <> struct Load<DFS> {
  typedef df2 Z;
  static __device__ __forceinline__ Z at(const void* p, size_t lo, size_t i) {
    return {((const float*)p)[i], ((const float*)p)[i + lo]};
  }
  static __device__ __forceinline__ Z zero() { return {0.f, 0.f}; }
};

// ---- arithmetic policies ----------------------------------------------------
// FP32 and FP64 mix the coupled columns at the four corners first ("node" mixing,
// 4 multiply-adds per term) and form the features once per row.
#define SG_NODE_MIX                                                                                  \
  struct State {                                                                                     \
    Acc a, b, c, d;                                                                                  \
  };                                                                                                 \
  static __device__ __forceinline__ void init(State& s) { s.a = s.b = s.c = s.d = zero(); }        \
  template <typename Z>                                                                              \
  static __device__ __forceinline__ void term(State& s, T w, Z za, Z zb, Z zc, Z zd) {              \
    fma(s.a, w, za);                                                                                 \
    fma(s.b, w, zb);                                                                                 \
    fma(s.c, w, zc);                                                                                 \
    fma(s.d, w, zd);                                                                                 \
  }                                                                                                  \
  static __device__ __forceinline__ void features(State& s, T& A, T& B, T& C) {                    \
    const T ta = get(s.a), tb = get(s.b), tc = get(s.c), td = get(s.d);                             \
    A = half(sub(ta, tc));                                                                           \
    B = half(sub(tb, td));                                                                           \
    C = sixth(sub(add(ta, tc), add(tb, td)));                                                        \
  }

struct ArF32 {
  static constexpr bool kUsesTable = false;
  typedef float T;
  typedef float Acc;
  static __device__ __forceinline__ T weight(const ApplyArgs& a, int k, size_t e, int t) {
    return a.c32[(size_t)k * a.Nc + e] * a.g32[t];
  }
  static __device__ __forceinline__ Acc zero() { return 0.f; }
  static __device__ __forceinline__ void fma(Acc& s, T w, float z) { s = fmaf(w, z, s); }
  static __device__ __forceinline__ void fma(Acc& s, T w, double z) { s = fmaf(w, (float)z, s); }
  static __device__ __forceinline__ void fma(Acc& s, T w, df2 z) { s = fmaf(w, z.hi, s); }
  static __device__ __forceinline__ T get(Acc s) { return s; }
  static __device__ __forceinline__ T add(T x, T y) { return x + y; }
  static __device__ __forceinline__ T sub(T x, T y) { return x - y; }
  static __device__ __forceinline__ T half(T x) { return 0.5f * x; }
  static __device__ __forceinline__ T sixth(T x) { return x * (1.f / 6.f); }
  static __device__ __forceinline__ void acc_add(Acc& s, T x) { s += x; }
  static __device__ __forceinline__ void acc_sub(Acc& s, T x) { s -= x; }
  SG_NODE_MIX
};

struct ArF64 {
  static constexpr bool kUsesTable = false;
  typedef double T;
  typedef double Acc;
  static __device__ __forceinline__ T weight(const ApplyArgs& a, int k, size_t e, int t) {
    return a.c64[(size_t)k * a.Nc + e] * a.g64[t];
  }
  static __device__ __forceinline__ Acc zero() { return 0.0; }
  static __device__ __forceinline__ void fma(Acc& s, T w, float z) { s = ::fma(w, (double)z, s); }
  static __device__ __forceinline__ void fma(Acc& s, T w, double z) { s = ::fma(w, z, s); }
  static __device__ __forceinline__ void fma(Acc& s, T w, df2 z) { s = ::fma(w, (double)z.hi + (double)z.lo, s); }
  static __device__ __forceinline__ T get(Acc s) { return s; }
  static __device__ __forceinline__ T add(T x, T y) { return x + y; }
  static __device__ __forceinline__ T sub(T x, T y) { return x - y; }
  static __device__ __forceinline__ T half(T x) { return 0.5 * x; }
  static __device__ __forceinline__ T sixth(T x) { return x / 6.0; }
  static __device__ __forceinline__ void acc_add(Acc& s, T x) { s += x; }
  static __device__ __forceinline__ void acc_sub(Acc& s, T x) { s -= x; }
  SG_NODE_MIX
};

struct ArDF {
  typedef df2 T;
  typedef dacc Acc;
  // with the weight table, k is the term's weight slot (precomputed c_k(e) gamma products)
  static constexpr bool kUsesTable = true;
  static __device__ __forceinline__ T weight(const ApplyArgs& a, int k, size_t e, int t) {
    if (a.wdf) return a.wdf[(size_t)k * a.Nc + e];
    return df_mul(a.cdf[(size_t)k * a.Nc + e], a.gdf[t]);
  }
  static __device__ __forceinline__ Acc zero() { return dacc_zero(); }
  static __device__ __forceinline__ void fma(Acc& s, T w, float z) { dacc_fma(s, w, z); }
  static __device__ __forceinline__ void fma(Acc& s, T w, df2 z) { dacc_fma(s, w, z); }
  static __device__ __forceinline__ void fma(Acc& s, T w, double z) { dacc_fma(s, w, df_from_double(z)); }
  static __device__ __forceinline__ T get(Acc s) { return dacc_get(s); }
  static __device__ __forceinline__ T add(T x, T y) { return df_add(x, y); }
  static __device__ __forceinline__ T sub(T x, T y) { return df_sub(x, y); }
  static __device__ __forceinline__ T half(T x) { return df_scale2(x, 0.5f); }
  static __device__ __forceinline__ T sixth(T x) {
    const df2 s6 = {0.1666666716337204f, -4.967053879312289e-09f};   // 1/6 = hi + lo
    return df_mul(x, s6);
  }
  static __device__ __forceinline__ void acc_add(Acc& s, T x) { dacc_add(s, x); }
  static __device__ __forceinline__ void acc_sub(Acc& s, T x) { dacc_sub(s, x); }

  // Double-float mixes the three cell features of each coupled column ("feature"
  // mixing): the features of an FP32/BF16 column are formed exactly with TwoSum, so
  // the rounding error of the mixed features is relative to the features themselves
  // (for smooth columns about h |grad| instead of |X|), which keeps the operator's
  // error far below the FP64-class tolerance of the outer Krylov method.
  struct State {
    dacc d1, d2, hg;
  };
  static __device__ __forceinline__ void init(State& s) { s.d1 = s.d2 = s.hg = dacc_zero(); }
  static __device__ __forceinline__ void term(State& s, T w, float za, float zb, float zc, float zd) {
    df2 f1, f2, f3;
    two_sum(za, -zc, f1.hi, f1.lo);                    // exact
    two_sum(zb, -zd, f2.hi, f2.lo);                    // exact
    float p, ep, q, eq;
    two_sum(za, zc, p, ep);
    two_sum(zb, zd, q, eq);
    float s3, e3;
    two_sum(p, -q, s3, e3);
    two_sum(s3, __fadd_rn(e3, __fsub_rn(ep, eq)), f3.hi, f3.lo);
    dacc_fma(s.d1, w, f1);
    dacc_fma(s.d2, w, f2);
    dacc_fma(s.hg, w, f3);
  }
  static __device__ __forceinline__ df2 dsub(df2 a, df2 b) {
    float s, e;
    two_sum(a.hi, -b.hi, s, e);
    e = __fadd_rn(e, __fsub_rn(a.lo, b.lo));
    df2 r;
    two_sum(s, e, r.hi, r.lo);
    return r;
  }
  static __device__ __forceinline__ void term(State& s, T w, df2 za, df2 zb, df2 zc, df2 zd) {
    dacc_fma(s.d1, w, dsub(za, zc));
    dacc_fma(s.d2, w, dsub(zb, zd));
    dacc h = dacc_from(za);
    dacc_add(h, zc);
    dacc_sub(h, zb);
    dacc_sub(h, zd);
    dacc_fma(s.hg, w, dacc_get(h));
  }
  static __device__ __forceinline__ void term(State& s, T w, double za, double zb, double zc, double zd) {
    term(s, w, df_from_double(za), df_from_double(zb), df_from_double(zc), df_from_double(zd));
  }
  static __device__ __forceinline__ void features(State& s, T& A, T& B, T& C) {
    A = half(dacc_get(s.d1));
    B = half(dacc_get(s.d2));
    C = sixth(dacc_get(s.hg));
  }
};

// ---- output / epilogue -------------------------------------------------------
template <typename TS> struct Store;
template <> struct Store<double> {
  static __device__ __forceinline__ void put(void* p, size_t, size_t i, double v) { ((double*)p)[i] = v; }
  static __device__ __forceinline__ void put(void* p, size_t, size_t i, float v) { ((double*)p)[i] = v; }
  static __device__ __forceinline__ void put(void* p, size_t, size_t i, df2 v) { ((double*)p)[i] = df_to_double(v); }
};
template <> struct Store<float> {
  static __device__ __forceinline__ void put(void* p, size_t, size_t i, double v) { ((float*)p)[i] = (float)v; }
  static __device__ __forceinline__ void put(void* p, size_t, size_t i, float v) { ((float*)p)[i] = v; }
  static __device__ __forceinline__ void put(void* p, size_t, size_t i, df2 v) { ((float*)p)[i] = v.hi; }
};
template <> struct Store<bf16> {
  static __device__ __forceinline__ void put(void* p, size_t, size_t i, double v) { ((bf16*)p)[i] = __float2bfloat16_rn((float)v); }
  static __device__ __forceinline__ void put(void* p, size_t, size_t i, float v) { ((bf16*)p)[i] = __float2bfloat16_rn(v); }
  static __device__ __forceinline__ void put(void* p, size_t, size_t i, df2 v) { ((bf16*)p)[i] = __float2bfloat16_rn(v.hi); }
};
template <> struct Store<DFS> {
  static __device__ __forceinline__ void put(void* p, size_t lo, size_t i, df2 v) {
    ((float*)p)[i] = v.hi;
    ((float*)p)[i + lo] = v.lo;
  }
  static __device__ __forceinline__ void put(void* p, size_t lo, size_t i, double v) { put(p, lo, i, df_from_double(v)); }
  static __device__ __forceinline__ void put(void* p, size_t lo, size_t i, float v) { put(p, lo, i, df2{v, 0.f}); }
};

// R - y in the policy's arithmetic (R stored as TR)
struct NoR {};
template <class AR, typename TR> struct Epi {
  template <typename T> static __device__ __forceinline__ T f(const void*, size_t, size_t, T y) { return y; }
};
template <> struct Epi<ArF32, double> {
  static __device__ __forceinline__ float f(const void* R, size_t, size_t i, float y) { return (float)((const double*)R)[i] - y; }
};
template <> struct Epi<ArF32, DFS> {
  static __device__ __forceinline__ float f(const void* R, size_t, size_t i, float y) { return ((const float*)R)[i] - y; }
};
template <> struct Epi<ArF32, float> {
  static __device__ __forceinline__ float f(const void* R, size_t, size_t i, float y) { return ((const float*)R)[i] - y; }
};
template <> struct Epi<ArF64, double> {
  static __device__ __forceinline__ double f(const void* R, size_t, size_t i, double y) { return ((const double*)R)[i] - y; }
};
template <> struct Epi<ArDF, DFS> {
  static __device__ __forceinline__ df2 f(const void* R, size_t lo, size_t i, df2 y) {
    return df_sub(df2{((const float*)R)[i], ((const float*)R)[i + lo]}, y);
  }
};
template <> struct Epi<ArDF, double> {
  static __device__ __forceinline__ df2 f(const void* R, size_t, size_t i, df2 y) {
    return df_sub(df_from_double(((const double*)R)[i]), y);
  }
};

template <class AR, typename TXS, typename TYS, typename TRS>
__global__ void __launch_bounds__(NT) k_apply(ApplyArgs a) {
  typedef typename AR::T T;
  typedef typename AR::Acc Acc;
  typedef Load<TXS> LX;
  __shared__ T sA[NT], sB[NT], sC[NT];
  const int tid = threadIdx.x;
  const int tile = blockIdx.x / a.ngroups, group = blockIdx.x % a.ngroups;
  const int X0 = (tile % a.tiles_x) * OXN, Y0 = (tile / a.tiles_x) * OYN;   // first interior node of the tile
  const int cx = X0 + (tid % CXN), cy = Y0 + (tid / CXN);                   // this thread's cell
  const int n = a.n, m = a.m;
  const bool cell_ok = cx <= n - 2 && cy <= n - 2;
  const size_t e = (size_t)cx + (size_t)cy * (n - 1);
  // corner vertices: a = (cx, cy), b = (cx+1, cy), c = (cx+1, cy+1), d = (cx, cy+1)
  const bool ina = cx >= 1 && cx <= n - 2 && cy >= 1 && cy <= n - 2;
  const bool inb = cx + 1 <= n - 2 && cy >= 1 && cy <= n - 2;
  const bool inc = cx + 1 <= n - 2 && cy + 1 <= n - 2;
  const bool ind = cx >= 1 && cx <= n - 2 && cy + 1 <= n - 2;
  const long ia = (long)(cx - 1) + (long)(cy - 1) * m;   // interior index of corner a (may be < 0 when unused)
  const int rbeg = a.row0 + group * ROWS;
  const int rend = min(rbeg + ROWS, a.row0 + a.nrows);
  const int ox = tid % OXN, oy = tid / OXN;
  // stage the coupling terms of this CTA's rows in shared memory (one round trip instead of
  // one per term): column j and mode k
  __shared__ int s_tj[ROWS * MAXT], s_tk[ROWS * MAXT];
  const int tall0 = a.row_ptr[rbeg], tall1 = a.row_ptr[rend];
  const bool staged = tall1 - tall0 <= ROWS * MAXT;
  if (staged) {
    for (int t = tall0 + tid; t < tall1; t += NT) {
      s_tj[t - tall0] = a.tj[t];
      s_tk[t - tall0] = (AR::kUsesTable && a.wdf) ? a.ws[t] : a.tk[t];
    }
    __syncthreads();
  }
  for (int i = rbeg; i < rend; ++i) {
    const int t0 = a.row_ptr[i], t1 = a.row_ptr[i + 1];
    typename AR::State st;
    AR::init(st);
    if (cell_ok) {
#pragma unroll 2
      for (int t = t0; t < t1; ++t) {
        const int jj = staged ? s_tj[t - tall0] : a.tj[t];
        const int kk = staged ? s_tk[t - tall0] : ((AR::kUsesTable && a.wdf) ? a.ws[t] : a.tk[t]);
        const size_t base = (size_t)jj * a.Nx;
        const T w = AR::weight(a, kk, e, t);
        const typename LX::Z za = ina ? LX::at(a.X, a.xlo, base + ia) : LX::zero();
        const typename LX::Z zb = inb ? LX::at(a.X, a.xlo, base + ia + 1) : LX::zero();
        const typename LX::Z zc = inc ? LX::at(a.X, a.xlo, base + ia + 1 + m) : LX::zero();
        const typename LX::Z zd = ind ? LX::at(a.X, a.xlo, base + ia + m) : LX::zero();
        AR::term(st, w, za, zb, zc, zd);
      }
    }
    AR::features(st, sA[tid], sB[tid], sC[tid]);
    __syncthreads();
    if (tid < OXN * OYN) {
      const int ix = X0 + ox, iy = Y0 + oy;
      if (ix < m && iy < m) {
        const int cSWn = ox + oy * CXN;          // cell SW of the node: node is its NE corner (c)
        const int cSEn = cSWn + 1;               // node is its NW corner (d)
        const int cNWn = cSWn + CXN;             // node is its SE corner (b)
        const int cNEn = cSWn + CXN + 1;         // node is its SW corner (a)
        Acc y = AR::zero();
        AR::acc_add(y, sA[cNEn]);
        AR::acc_add(y, sC[cNEn]);
        AR::acc_add(y, sB[cNWn]);
        AR::acc_sub(y, sC[cNWn]);
        AR::acc_add(y, sC[cSWn]);
        AR::acc_sub(y, sA[cSWn]);
        AR::acc_sub(y, sB[cSEn]);
        AR::acc_sub(y, sC[cSEn]);
        const size_t s = (size_t)ix + (size_t)iy * m;
        const T out = Epi<AR, TRS>::f(a.R, a.rlo, (size_t)(i - a.rbase) * a.Nx + s, AR::get(y));
        Store<TYS>::put(a.Y, a.ylo, (size_t)(i - a.ybase) * a.Nx + s, out);
      }
    }
    __syncthreads();
  }
}

template <class AR, typename TXS, typename TYS, typename TRS>
int launch_t(sg_ctx* h, ApplyArgs& a) {
  const int tiles_y = (h->m + OYN - 1) / OYN;
  a.tiles_x = (h->m + OXN - 1) / OXN;
  a.ngroups = (a.nrows + ROWS - 1) / ROWS;
  const unsigned grid = (unsigned)a.ngroups * (unsigned)(a.tiles_x * tiles_y);
  k_apply<AR, TXS, TYS, TRS><<<grid, NT, 0, h->stream>>>(a);
  SG_CUDA(h, cudaGetLastError());
  count_launch(h);
  return SG_OK;
}

template <class AR, typename TXS, typename TYS>
int pick_r(sg_ctx* h, ApplyArgs& a, int rprec) {
  if (!a.R) return launch_t<AR, TXS, TYS, NoR>(h, a);
  if (rprec == SG_F64) return launch_t<AR, TXS, TYS, double>(h, a);
  if (rprec == SG_F32) {
    if constexpr (std::is_same<AR, ArF32>::value) return launch_t<AR, TXS, TYS, float>(h, a);
  }
  if (rprec == SG_DF64) {
    if constexpr (!std::is_same<AR, ArF64>::value) return launch_t<AR, TXS, TYS, DFS>(h, a);
  }
  return sg_fail(h, SG_E_ARG, "apply: unsupported residual precision");
}

template <class AR, typename TXS>
int pick_y(sg_ctx* h, ApplyArgs& a, int yprec, int rprec) {
  switch (yprec) {
    case SG_F64: return pick_r<AR, TXS, double>(h, a, rprec);
    case SG_F32: return pick_r<AR, TXS, float>(h, a, rprec);
    case SG_BF16: return pick_r<AR, TXS, bf16>(h, a, rprec);
    case SG_DF64:
      if constexpr (std::is_same<AR, ArDF>::value) return pick_r<AR, TXS, DFS>(h, a, rprec);
      break;
  }
  return sg_fail(h, SG_E_ARG, "apply: unsupported output precision");
}

template <class AR>
int pick_x(sg_ctx* h, ApplyArgs& a, int xprec, int yprec, int rprec) {
  switch (xprec) {
    case SG_F64: return pick_y<AR, double>(h, a, yprec, rprec);
    case SG_F32: return pick_y<AR, float>(h, a, yprec, rprec);
    case SG_BF16: return pick_y<AR, bf16>(h, a, yprec, rprec);
    case SG_DF64:
      if constexpr (!std::is_same<AR, ArF64>::value) return pick_y<AR, DFS>(h, a, yprec, rprec);
      break;
  }
  return sg_fail(h, SG_E_ARG, "apply: unsupported input precision");
}
}  // namespace

int launch_apply(sg_ctx* h, int which, int xprec, const void* X, size_t xlo, int yprec, void* Y, size_t ylo,
                 int rprec, const void* R, size_t rlo, int row0, int nrows, int ybase, int rbase, int arith) {
  if (nrows <= 0) return SG_OK;
  const TermTable& T = which == 0   ? h->t_all
                       : which == 1 ? h->t_lower
                       : which == 2 ? h->t_upper
                       : which == 3 ? h->t_off
                                    : h->t_diag;
  ApplyArgs a{};
  a.X = X, a.xlo = xlo, a.Y = Y, a.ylo = ylo, a.R = R, a.rlo = rlo;
  a.c64 = h->coef64, a.c32 = h->coef32, a.cdf = (const df2*)h->coefdf;
  a.wdf = (const df2*)h->wdf, a.ws = T.ws;
  a.row_ptr = T.row_ptr, a.tj = T.j, a.tk = T.k, a.g64 = T.g, a.g32 = T.gf, a.gdf = (const df2*)T.gdf;
  a.row0 = row0, a.nrows = nrows, a.ybase = ybase, a.rbase = rbase, a.n = h->n, a.m = h->m;
  a.Nx = h->Nx, a.Nc = h->Nc;
  if (arith == SG_F64) return pick_x<ArF64>(h, a, xprec, yprec, rprec);
  if (arith == SG_DF64) return pick_x<ArDF>(h, a, xprec, yprec, rprec);
  return pick_x<ArF32>(h, a, xprec, yprec, rprec);
}
