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
// One lane per cell: a warp owns 32 consecutive cells of a cell row and walks up a
// strip of cell rows for one output row i.  Per cell row and coupling it loads the two
// right-hand corners of its cell (the left ones come from the neighbouring lane by a
// shuffle), forms the cell's features, and then finishes the node on its cell's SW
// corner from the features of the four cells around it: the two of this lane (this cell
// row and the previous one, kept in registers) and the two of the lane on its left,
// which sends their combined contribution in one shuffle.  Lane 0 only supplies its
// cell to lane 1, so warps advance by 31 cells.  No shared memory, no block barriers
// in the main loop; the coupling table of the row is staged in shared memory once.
//
// Arithmetic policies: FP32, FP64 (IEEE double) and DF (double-float, see df64.cuh;
// used where FP64-class accuracy is needed at FP32 throughput).
#include <type_traits>

#include "df64.cuh"
#include "sg_internal.h"

namespace {
constexpr int WARPS = 8, NT = 32 * WARPS;          // warps per CTA (all on the same output row)
constexpr int STRIP_DEFAULT = 16;                   // node rows per warp strip (tunable: sg_autotune)
constexpr int MAXT = 40;                            // coupling terms per row: at most 1 + 2M (M <= 16 at set-up)

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
  const double* w64;   // optional table of the same weights in FP64
  const int* ws;       // weight slot of each term
  const unsigned* qmax; // SG_F32Q input: block maxima of X (its grid scales)
  const int* row_ptr;
  const int* tj;
  const int* tk;
  const double* g64;
  const float* g32;
  const df2* gdf;
  int row0, nrows, ybase, rbase, n, m;
  size_t Nx, Nc;
  int nwx, nstrips, strip;   // warp columns (31 cells each), strips per output row, node rows per strip
  int unit0;                 // every row's first term is the mean coupling with weight exactly 1
};

// ---- storage access --------------------------------------------------------
struct DFS {};   // tag: double-float storage, hi array at p, lo array at p + lo

// ldq: the element at p as the policy's input type when ok, else zero (nothing is read when ok is false)
template <typename TS> struct Load;
template <> struct Load<double> {
  typedef double Z;
  typedef double E;                                  // stored element
  static __device__ __forceinline__ Z ldq(const E* p, size_t, bool ok) { return ok ? __ldg(p) : 0.0; }
  static __device__ __forceinline__ Z zero() { return 0.0; }
};
template <> struct Load<float> {
  typedef float Z;
  typedef float E;
  static __device__ __forceinline__ Z ldq(const E* p, size_t, bool ok) { return ok ? __ldg(p) : 0.f; }
  static __device__ __forceinline__ Z zero() { return 0.f; }
};
template <> struct Load<bf16> {
  typedef float Z;
  typedef bf16 E;
  static __device__ __forceinline__ Z ldq(const E* p, size_t, bool ok) { return ok ? __bfloat162float(__ldg(p)) : 0.f; }
  static __device__ __forceinline__ Z zero() { return 0.f; }
};
// FP32 storage read through per-block fixed-point grids (SG_F32Q): the kernel turns each loaded value
// into the biased integer fma(z, s_j, 1.5 2^23) of its grid value and scales the coupling's weight by
// the block's quantum, so the double-float policy forms its cell features by plain FP32 differences,
// which are exact for such values
struct QF32 {};
struct qf {
  float v;
};
template <> struct Load<QF32> {
  typedef qf Z;
  typedef float E;
  static __device__ __forceinline__ Z ldq(const E* p, size_t, bool ok) { return qf{ok ? __ldg(p) : 0.f}; }
  static __device__ __forceinline__ Z zero() { return qf{0.f}; }
};
template <> struct Load<DFS> {
  typedef df2 Z;
  typedef float E;                                   // hi array; the lo array follows at + lo
  static __device__ __forceinline__ Z ldq(const E* p, size_t lo, bool ok) {
    return ok ? Z{__ldg(p), __ldg(p + lo)} : Z{0.f, 0.f};
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
  static __host__ __device__ __forceinline__ const void* table(const ApplyArgs&) { return nullptr; }
  static constexpr int kUnroll = 4;        // couplings in flight per step (latency-bound stage updates)
  typedef float T;
  typedef float Acc;
  typedef float G;
  typedef float CE;                        // coefficient element
  static __device__ __forceinline__ G gval(const ApplyArgs& a, int t) { return a.g32[t]; }
  template <bool WT> static __device__ __forceinline__ const CE* cbase(const ApplyArgs& a) { return a.c32; }
  template <bool WT> static __device__ __forceinline__ T weight(CE c, G g) { return c * g; }
  static __device__ __forceinline__ Acc zero() { return 0.f; }
  static __device__ __forceinline__ T wzero() { return 0.f; }
  static __device__ __forceinline__ void fma(Acc& s, T w, float z) { s = fmaf(w, z, s); }
  static __device__ __forceinline__ void fma(Acc& s, T w, double z) { s = fmaf(w, (float)z, s); }
  static __device__ __forceinline__ void fma(Acc& s, T w, df2 z) { s = fmaf(w, z.hi, s); }
  static __device__ __forceinline__ T get(Acc s) { return s; }
  static __device__ __forceinline__ T get_raw(Acc s) { return s; }
  static __device__ __forceinline__ Acc acc_from(T x) { return x; }
  static __device__ __forceinline__ T add(T x, T y) { return x + y; }
  static __device__ __forceinline__ T sub(T x, T y) { return x - y; }
  static __device__ __forceinline__ T half(T x) { return 0.5f * x; }
  static __device__ __forceinline__ T sixth(T x) { return x * (1.f / 6.f); }
  static __device__ __forceinline__ void acc_add(Acc& s, T x) { s += x; }
  static __device__ __forceinline__ void acc_sub(Acc& s, T x) { s -= x; }
  SG_NODE_MIX
};

struct ArF64 {
  // with the weight table, the element is the FP64 product c_k(e) gamma of the term's slot (the
  // same value the product below forms)
  static constexpr bool kUsesTable = true;
  static constexpr int kUnroll = 2;
  typedef double T;
  typedef double Acc;
  typedef double G;
  typedef double CE;
  static __host__ __device__ __forceinline__ const void* table(const ApplyArgs& a) { return a.w64; }
  static __device__ __forceinline__ G gval(const ApplyArgs& a, int t) { return a.g64[t]; }
  template <bool WT> static __device__ __forceinline__ const CE* cbase(const ApplyArgs& a) { return WT ? a.w64 : a.c64; }
  template <bool WT> static __device__ __forceinline__ T weight(CE c, G g) { return WT ? c : c * g; }
  static __device__ __forceinline__ Acc zero() { return 0.0; }
  static __device__ __forceinline__ T wzero() { return 0.0; }
  static __device__ __forceinline__ void fma(Acc& s, T w, float z) { s = ::fma(w, (double)z, s); }
  static __device__ __forceinline__ void fma(Acc& s, T w, double z) { s = ::fma(w, z, s); }
  static __device__ __forceinline__ void fma(Acc& s, T w, df2 z) { s = ::fma(w, (double)z.hi + (double)z.lo, s); }
  static __device__ __forceinline__ T get(Acc s) { return s; }
  static __device__ __forceinline__ T get_raw(Acc s) { return s; }
  static __device__ __forceinline__ Acc acc_from(T x) { return x; }
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
  static constexpr int kUnroll = 2;
  static __host__ __device__ __forceinline__ const void* table(const ApplyArgs& a) { return a.wdf; }
  typedef df2 G;
  typedef df2 CE;
  static __device__ __forceinline__ G gval(const ApplyArgs& a, int t) { return a.gdf[t]; }
  // WT: with the table, the element is the precomputed product c_k(e) gamma of the term's slot
  template <bool WT> static __device__ __forceinline__ const CE* cbase(const ApplyArgs& a) { return WT ? a.wdf : a.cdf; }
  template <bool WT> static __device__ __forceinline__ T weight(CE c, G g) { return WT ? c : df_mul(c, g); }
  static __device__ __forceinline__ Acc zero() { return dacc_zero(); }
  static __device__ __forceinline__ T wzero() { return {0.f, 0.f}; }
  static __device__ __forceinline__ void fma(Acc& s, T w, float z) { dacc_fma(s, w, z); }
  static __device__ __forceinline__ void fma(Acc& s, T w, df2 z) { dacc_fma(s, w, z); }
  static __device__ __forceinline__ void fma(Acc& s, T w, double z) { dacc_fma(s, w, df_from_double(z)); }
  static __device__ __forceinline__ T get(Acc s) { return dacc_get(s); }
  // the pair (s, c) without the final TwoSum: hi + lo is still the value (|c| is a few ulp of s), which
  // is all a further compensated sum or an FP64 store needs
  static __device__ __forceinline__ T get_raw(Acc s) { return {s.s, s.c}; }
  static __device__ __forceinline__ Acc acc_from(T x) { return dacc_from(x); }
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
  // biased grid integers (SG_F32Q): 1.5 2^23 + k with |k| < 2^22, so the two differences
  // (< 2^23) and the alternating sum (< 2^24) are integers that FP32 holds exactly, and so are
  // their products with the block's quantum q (a power of two, at least 2^-107): the exact features
  static __device__ __forceinline__ void qterm(State& s, T w, float za, float zb, float zc, float zd, float q) {
    const float f1 = __fmul_rn(__fsub_rn(za, zc), q);
    const float f2 = __fmul_rn(__fsub_rn(zb, zd), q);
    const float f3 = __fmul_rn(__fadd_rn(__fsub_rn(za, zb), __fsub_rn(zc, zd)), q);
    dacc_fma(s.d1, w, f1);
    dacc_fma(s.d2, w, f2);
    dacc_fma(s.hg, w, f3);
  }
  // qterm with the weight exactly 1 on zero sums: the features themselves, no rounding error
  static __device__ __forceinline__ void qterm_unit(State& s, float za, float zb, float zc, float zd, float q) {
    s.d1 = {__fmul_rn(__fsub_rn(za, zc), q), 0.f};
    s.d2 = {__fmul_rn(__fsub_rn(zb, zd), q), 0.f};
    s.hg = {__fmul_rn(__fadd_rn(__fsub_rn(za, zb), __fsub_rn(zc, zd)), q), 0.f};
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
    A = half(get_raw(s.d1));       // consumed only by compensated sums: no renormalisation needed
    B = half(get_raw(s.d2));
    C = sixth(get_raw(s.hg));
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

// R - y in the policy's arithmetic (R stored as TR).  ld() fetches R's value early (the
// kernel issues it before the coupling loads so its latency overlaps them), f() combines.
struct NoR {};
template <class AR, typename TR> struct Epi {
  typedef int Raw;
  static __device__ __forceinline__ Raw ld(const void*, size_t, size_t) { return 0; }
  template <typename T> static __device__ __forceinline__ T f(Raw, T y) { return y; }
};
template <> struct Epi<ArF32, double> {
  typedef double Raw;
  static __device__ __forceinline__ Raw ld(const void* R, size_t, size_t i) { return ((const double*)R)[i]; }
  static __device__ __forceinline__ float f(Raw r, float y) { return (float)r - y; }
};
template <> struct Epi<ArF32, DFS> {
  typedef float Raw;
  static __device__ __forceinline__ Raw ld(const void* R, size_t, size_t i) { return ((const float*)R)[i]; }
  static __device__ __forceinline__ float f(Raw r, float y) { return r - y; }
};
template <> struct Epi<ArF32, float> {
  typedef float Raw;
  static __device__ __forceinline__ Raw ld(const void* R, size_t, size_t i) { return ((const float*)R)[i]; }
  static __device__ __forceinline__ float f(Raw r, float y) { return r - y; }
};
template <> struct Epi<ArF64, double> {
  typedef double Raw;
  static __device__ __forceinline__ Raw ld(const void* R, size_t, size_t i) { return ((const double*)R)[i]; }
  static __device__ __forceinline__ double f(Raw r, double y) { return r - y; }
};
template <> struct Epi<ArDF, DFS> {
  typedef df2 Raw;
  static __device__ __forceinline__ Raw ld(const void* R, size_t lo, size_t i) {
    return df2{((const float*)R)[i], ((const float*)R)[i + lo]};
  }
  static __device__ __forceinline__ df2 f(Raw r, df2 y) { return df_sub(r, y); }
};
template <> struct Epi<ArDF, double> {
  typedef double Raw;
  static __device__ __forceinline__ Raw ld(const void* R, size_t, size_t i) { return ((const double*)R)[i]; }
  static __device__ __forceinline__ df2 f(Raw r, df2 y) { return df_sub(df_from_double(r), y); }
};

__device__ __forceinline__ float shfl_up1(float v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_up1(double v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ df2 shfl_up1(df2 v) {
  return {__shfl_up_sync(0xffffffffu, v.hi, 1), __shfl_up_sync(0xffffffffu, v.lo, 1)};
}

__device__ __forceinline__ float ldg_ce(const float* p) { return __ldg(p); }
__device__ __forceinline__ double ldg_ce(const double* p) { return __ldg(p); }
__device__ __forceinline__ df2 ldg_ce(const df2* p) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return {v.x, v.y};
}

// The row's couplings as shared-memory tables: the coupled column's base pointer, the base
// pointer of its weight row (mode k, or table slot), and the coupling value.
template <class AR, typename XE> struct RowTerms {
  const XE* xp[MAXT];
  const typename AR::CE* wp[MAXT];
  typename AR::G g[MAXT];
  float qs[MAXT], qq[MAXT];        // SG_F32Q: grid scale and quantum of the coupled column's block
};

template <class AR, bool WT, typename TXS, typename TYS, typename TRS>
__global__ void __launch_bounds__(NT) k_apply(ApplyArgs a) {
  typedef typename AR::T T;
  typedef typename AR::Acc Acc;
  typedef Load<TXS> LX;
  typedef typename LX::Z Z;
  typedef Epi<AR, TRS> E;
  typedef typename LX::E XE;
  __shared__ RowTerms<AR, XE> rt;
  // rows vary fastest across the grid, so every row's CTAs over one grid tile run close together
  // and the coupled columns' tile is read from HBM once and then from L2
  const int i = a.row0 + blockIdx.x;                       // output row of this CTA
  const int t0 = a.row_ptr[i];
  const int nt = a.row_ptr[i + 1] - t0;                    // <= MAXT (M <= 16 at set-up)
  for (int t = threadIdx.x; t < nt; t += NT) {
    rt.xp[t] = (const XE*)a.X + (size_t)a.tj[t0 + t] * a.Nx;
    rt.wp[t] = AR::template cbase<WT>(a) + (size_t)(WT ? a.ws[t0 + t] : a.tk[t0 + t]) * a.Nc;
    rt.g[t] = AR::gval(a, t0 + t);
    if constexpr (std::is_same<TXS, QF32>::value) {
      const unsigned mb = a.qmax[a.tj[t0 + t]];
      rt.qs[t] = qgrid_scale(mb), rt.qq[t] = qgrid_quantum(mb);
    }
  }
  __syncthreads();
  const int gw = blockIdx.y * WARPS + (threadIdx.x >> 5);
  if (gw >= a.nwx * a.nstrips) return;                     // whole warps only
  const int lane = threadIdx.x & 31;
  const int n = a.n, m = a.m;
  const size_t xlo = a.xlo;
  const int cx = 31 * (gw % a.nwx) + lane;                 // cell column = vertex column of its SW corner
  const int cy0 = a.strip * (gw / a.nwx);                  // first cell row (primes the window)
  const int cy1 = min(cy0 + a.strip, n - 2);               // last cell row = last node row of the strip
  const bool okl = cx >= 1 && cx <= n - 2;                 // left corners (vertex column cx) interior
  const bool okr = cx + 1 <= n - 2;                        // right corners (vertex column cx + 1) interior
  const bool node_col = lane >= 1 && cx <= n - 2;          // this lane finishes node (cx, cy)
  const int cxw = min(cx, n - 2);                          // weight column (cells beyond the grid have zero corners)
  typename E::Raw rv;
  T Ap = AR::wzero(), Bp = AR::wzero(), Cp = AR::wzero();   // features of cell (cx, cy - 1)
  for (int cy = cy0; cy <= cy1; ++cy) {
    const bool out = node_col && cy > cy0;                 // node (cx, cy): 1 <= cy <= n - 2 here
    const int s_node = (cx - 1) + (cy - 1) * m;            // interior index of vertex (cx, cy) (< 2^31)
    if (out) rv = E::ld(a.R, a.rlo, (size_t)(i - a.rbase) * a.Nx + s_node);
    const bool lo_ok = cy >= 1, hi_ok = cy + 1 <= n - 2;
    const bool oka = okl && lo_ok, okb = okr && lo_ok, okc = okr && hi_ok, okd = okl && hi_ok;
    const int e = cxw + cy * (n - 1);
    typename AR::State st;
    AR::init(st);
    int t = 0;
    if constexpr (std::is_same<AR, ArDF>::value && std::is_same<TXS, QF32>::value) {
      if (a.unit0 && nt > 0) {
        // the mean coupling: weight 1, so its exact grid features start the compensated sums as they
        // are (the same values the general step would give, without its weight load and products)
        const XE* p = rt.xp[0] + s_node;
        const float sq = rt.qs[0];
        const Z za = LX::ldq(p, xlo, oka), zb = LX::ldq(p + 1, xlo, okb);
        const Z zc = LX::ldq(p + 1 + m, xlo, okc), zd = LX::ldq(p + m, xlo, okd);
        AR::qterm_unit(st, __fmaf_rn(za.v, sq, SG_QBIAS), __fmaf_rn(zb.v, sq, SG_QBIAS),
                       __fmaf_rn(zc.v, sq, SG_QBIAS), __fmaf_rn(zd.v, sq, SG_QBIAS), rt.qq[0]);
        t = 1;
      }
    }
#pragma unroll AR::kUnroll
    for (; t < nt; ++t) {
      const XE* p = rt.xp[t] + s_node;                     // vertex (cx, cy) of column j
      const T w = AR::template weight<WT>(ldg_ce(rt.wp[t] + e), rt.g[t]);
      const Z za = LX::ldq(p, xlo, oka);
      const Z zb = LX::ldq(p + 1, xlo, okb);
      const Z zc = LX::ldq(p + 1 + m, xlo, okc);
      const Z zd = LX::ldq(p + m, xlo, okd);
      if constexpr (std::is_same<TXS, QF32>::value) {
        const float sq = rt.qs[t];                         // exact: the product is rounded once, to an integer
        AR::qterm(st, w, __fmaf_rn(za.v, sq, SG_QBIAS), __fmaf_rn(zb.v, sq, SG_QBIAS), __fmaf_rn(zc.v, sq, SG_QBIAS),
                  __fmaf_rn(zd.v, sq, SG_QBIAS), rt.qq[t]);
      } else {
        AR::term(st, w, za, zb, zc, zd);
      }
    }
    T Ac, Bc, Cc;
    AR::features(st, Ac, Bc, Cc);
    if (cy > cy0) {
      // this lane's cells seen from node (cx + 1, cy): SE corner of cell (cx, cy) and NE corner of
      // cell (cx, cy - 1); sent to the right neighbour
      Acc u = AR::acc_from(Bc);
      AR::acc_sub(u, Cc);
      AR::acc_add(u, Cp);
      AR::acc_sub(u, Ap);
      const T ul = shfl_up1(AR::get_raw(u));
      if (out) {
        // node (cx, cy): SW corner of cell (cx, cy), NW corner of cell (cx, cy - 1), plus the left lane
        Acc y = AR::acc_from(Ac);
        AR::acc_add(y, Cc);
        AR::acc_sub(y, Bp);
        AR::acc_sub(y, Cp);
        AR::acc_add(y, ul);
        // an FP64 store rounds hi + lo once either way; other outputs take the renormalised pair
        const T yv = std::is_same<TYS, double>::value ? AR::get_raw(y) : AR::get(y);
        Store<TYS>::put(a.Y, a.ylo, (size_t)(i - a.ybase) * a.Nx + s_node, E::f(rv, yv));
      }
    }
    Ap = Ac, Bp = Bc, Cp = Cc;
  }
}

// FP32 arithmetic, two cells per lane.  Lane l of a warp owns the cells cx0 = X + 2l and cx0 + 1
// of each cell row (X = 62 w, even, so the cells' coefficient pair is one aligned 8-byte load) and
// walks a strip of cell rows for one output row i.  Per cell row and coupling it loads its two node
// columns in the two node rows of the cell row (the third column, cx0 + 2, comes from the right lane
// by a shuffle), loads the two cells' coefficients as one 8-byte pair (the cell rows have an even
// length) and mixes the corners with four multiply-adds per cell.  It finishes node cx0 + 1 from its
// own two cells in this and the previous cell row, and node cx0 from its first cell and the left
// lane's second cell, whose contribution arrives in one shuffle.  The edge lanes only half count:
// lane 0 has no left lane (it finishes node X + 1 only) and lane 31 no right column (its second cell
// is incomplete, it finishes node X + 62 only), so warp w writes nodes 62 w + 1 .. 62 w + 62 once
// each with no extra loads.  About half the load and address instructions per coupling of the
// one-cell-per-lane kernel.
template <typename TXS, typename TYS, typename TRS>
__global__ void __launch_bounds__(NT, 4) k_apply_f32x2(ApplyArgs a) {
  typedef ArF32 AR;
  typedef Load<TXS> LX;
  typedef typename LX::E XE;
  typedef Epi<AR, TRS> E;
  __shared__ const XE* xp[MAXT];
  __shared__ const float* wp[MAXT];
  __shared__ float gg[MAXT];
  const int i = a.row0 + blockIdx.x;
  const int t0 = a.row_ptr[i];
  const int nt = a.row_ptr[i + 1] - t0;
  for (int t = threadIdx.x; t < nt; t += NT) {
    xp[t] = (const XE*)a.X + (size_t)a.tj[t0 + t] * a.Nx;
    wp[t] = a.c32 + (size_t)a.tk[t0 + t] * a.Nc;
    gg[t] = a.g32[t0 + t];
  }
  __syncthreads();
  const int gw = blockIdx.y * WARPS + (threadIdx.x >> 5);
  if (gw >= a.nwx * a.nstrips) return;
  const int lane = threadIdx.x & 31;
  const int n = a.n, m = a.m;
  const int cx0 = 62 * (gw % a.nwx) + 2 * lane;            // first cell (= vertex column of its SW corner)
  const int cy0 = a.strip * (gw / a.nwx);
  const int cy1 = min(cy0 + a.strip, n - 2);
  // columns cx0, cx0 + 1 interior?
  const bool ok0 = cx0 >= 1 && cx0 <= n - 2, ok1 = cx0 + 1 <= n - 2;
  const bool cellA = cx0 <= n - 2, cellB = cx0 + 1 <= n - 2;   // cells inside the grid of cells
  const bool outA = lane >= 1 && ok0, outB = lane <= 30 && ok1;   // nodes cx0, cx0 + 1 finished here
  const int cxw = min(cx0, n - 3);                             // weight pair (cells n - 3, n - 2 at most; n - 3 is even)
  // all lanes' node columns cx0, cx0 + 1 interior (first cell 62 w >= 1, last 62 w + 63 <= n - 2): uniform per warp
  const int wx0 = cx0 - 2 * lane;
  const bool inner = wx0 >= 1 && wx0 + 63 <= n - 2;
  const bool wshift = cxw != cx0;                              // only past the last cell pair (weights unused)
  float AAp = 0.f, BAp = 0.f, CAp = 0.f, ABp = 0.f, BBp = 0.f, CBp = 0.f;   // previous cell row's features
  typename E::Raw rvA{}, rvB{};
  for (int cy = cy0; cy <= cy1; ++cy) {
    const bool out_row = cy > cy0;
    const int sA = (cx0 - 1) + (cy - 1) * m;                   // interior index of vertex (cx0, cy)
    if (out_row) {
      if (outA) rvA = E::ld(a.R, a.rlo, (size_t)(i - a.rbase) * a.Nx + sA);
      if (outB) rvB = E::ld(a.R, a.rlo, (size_t)(i - a.rbase) * a.Nx + sA + 1);
    }
    const bool lo_ok = cy >= 1, hi_ok = cy + 1 <= n - 2;
    const int e = cxw + cy * (n - 1);
    float a0 = 0.f, b0 = 0.f, c0 = 0.f, d0 = 0.f;              // cell A corners mixed
    float a1 = 0.f, b1 = 0.f, c1 = 0.f, d1 = 0.f;              // cell B
    if (inner && lo_ok && hi_ok) {
      // every lane's corners are interior nodes in this cell row: no predicates, no selects
#pragma unroll 4
      for (int t = 0; t < nt; ++t) {
        const XE* p = xp[t] + sA;
        const float2 cw = __ldg(reinterpret_cast<const float2*>(wp[t] + e));
        const float g = gg[t];
        const float wA = cw.x * g, wB = cw.y * g;
        const float z0b = LX::ldq(p, 0, true), z1b = LX::ldq(p + 1, 0, true);
        const float z0t = LX::ldq(p + m, 0, true), z1t = LX::ldq(p + m + 1, 0, true);
        const float z2b = __shfl_down_sync(0xffffffffu, z0b, 1), z2t = __shfl_down_sync(0xffffffffu, z0t, 1);
        a0 = fmaf(wA, z0b, a0), b0 = fmaf(wA, z1b, b0), c0 = fmaf(wA, z1t, c0), d0 = fmaf(wA, z0t, d0);
        a1 = fmaf(wB, z1b, a1), b1 = fmaf(wB, z2b, b1), c1 = fmaf(wB, z2t, c1), d1 = fmaf(wB, z1t, d1);
      }
    } else {
#pragma unroll 4
      for (int t = 0; t < nt; ++t) {
        const XE* p = xp[t] + sA;
        const float2 cw = __ldg(reinterpret_cast<const float2*>(wp[t] + e));
        const float g = gg[t];
        const float wA = (wshift ? cw.y : cw.x) * g, wB = cw.y * g;
        const float z0b = LX::ldq(p, 0, ok0 && lo_ok), z1b = LX::ldq(p + 1, 0, ok1 && lo_ok);
        const float z0t = LX::ldq(p + m, 0, ok0 && hi_ok), z1t = LX::ldq(p + m + 1, 0, ok1 && hi_ok);
        const float z2b = __shfl_down_sync(0xffffffffu, z0b, 1), z2t = __shfl_down_sync(0xffffffffu, z0t, 1);
        a0 = fmaf(wA, z0b, a0), b0 = fmaf(wA, z1b, b0), c0 = fmaf(wA, z1t, c0), d0 = fmaf(wA, z0t, d0);
        a1 = fmaf(wB, z1b, a1), b1 = fmaf(wB, z2b, b1), c1 = fmaf(wB, z2t, c1), d1 = fmaf(wB, z1t, d1);
      }
    }
    // features; cells outside the grid of cells carry none
    float AA = cellA ? 0.5f * (a0 - c0) : 0.f, BA = cellA ? 0.5f * (b0 - d0) : 0.f;
    float CA = cellA ? ((a0 + c0) - (b0 + d0)) * (1.f / 6.f) : 0.f;
    float AB = cellB ? 0.5f * (a1 - c1) : 0.f, BB = cellB ? 0.5f * (b1 - d1) : 0.f;
    float CB = cellB ? ((a1 + c1) - (b1 + d1)) * (1.f / 6.f) : 0.f;
    if (out_row) {
      // cell B (this row and the previous one) seen from node cx0 + 2: sent to the right neighbour
      const float u = (BB - CB) + (CBp - ABp);
      const float ul = __shfl_up_sync(0xffffffffu, u, 1);
      const float yA = ((AA + CA) - (BAp + CAp)) + ul;                       // node (cx0, cy)
      const float yB = ((AB + CB) - (BBp + CBp)) + ((BA - CA) + (CAp - AAp));  // node (cx0 + 1, cy)
      if (outA) Store<TYS>::put(a.Y, a.ylo, (size_t)(i - a.ybase) * a.Nx + sA, E::f(rvA, yA));
      if (outB) Store<TYS>::put(a.Y, a.ylo, (size_t)(i - a.ybase) * a.Nx + sA + 1, E::f(rvB, yB));
    }
    AAp = AA, BAp = BA, CAp = CA, ABp = AB, BBp = BB, CBp = CB;
  }
}

template <class AR, typename TXS, typename TYS, typename TRS>
int launch_t(sg_ctx* h, ApplyArgs& a) {
  if constexpr (std::is_same<AR, ArF32>::value && !std::is_same<TXS, DFS>::value) {
    if (h->n >= 5) {
      a.nwx = (h->m + 61) / 62;                // warp w finishes nodes 62 w + 1 .. 62 w + 62
      long gy;
      for (;;) {
        a.nstrips = (h->m + a.strip - 1) / a.strip;
        gy = ((long)a.nwx * a.nstrips + WARPS - 1) / WARPS;
        if (gy <= 65535) break;
        a.strip *= 2;
      }
      k_apply_f32x2<TXS, TYS, TRS><<<dim3((unsigned)a.nrows, (unsigned)gy), NT, 0, h->stream>>>(a);
      SG_CUDA(h, cudaGetLastError());
      count_launch(h);
      return SG_OK;
    }
  }
  a.nwx = (h->m + 30) / 31;
  long gy;
  for (;;) {                                 // taller strips when the grid would exceed 65535 CTAs per row
    a.nstrips = (h->m + a.strip - 1) / a.strip;
    gy = ((long)a.nwx * a.nstrips + WARPS - 1) / WARPS;
    if (gy <= 65535) break;
    a.strip *= 2;
  }
  if (AR::kUsesTable && AR::table(a))
    k_apply<AR, true, TXS, TYS, TRS><<<dim3((unsigned)a.nrows, (unsigned)gy), NT, 0, h->stream>>>(a);
  else
    k_apply<AR, false, TXS, TYS, TRS><<<dim3((unsigned)a.nrows, (unsigned)gy), NT, 0, h->stream>>>(a);
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
    case SG_F32Q:
      if constexpr (std::is_same<AR, ArDF>::value) {
        if (yprec == SG_F64 && !a.R) return launch_t<AR, QF32, double, NoR>(h, a);
        if (yprec == SG_DF64 && !a.R) return launch_t<AR, QF32, DFS, NoR>(h, a);
      }
      break;
  }
  return sg_fail(h, SG_E_ARG, "apply: unsupported input precision");
}
}  // namespace

int launch_apply(sg_ctx* h, int which, int xprec, const void* X, size_t xlo, int yprec, void* Y, size_t ylo,
                 int rprec, const void* R, size_t rlo, int row0, int nrows, int ybase, int rbase, int arith) {
  if (h->elements == SG_P1)
    return launch_apply_p1(h, which, xprec, X, yprec, Y, rprec, R, row0, nrows, ybase, rbase, arith);
  if (nrows <= 0) return SG_OK;
  const TermTable& T = which == 0   ? h->t_all
                       : which == 1 ? h->t_lower
                       : which == 2 ? h->t_upper
                       : which == 3 ? h->t_off
                                    : h->t_diag;
  ApplyArgs a{};
  a.X = X, a.xlo = xlo, a.Y = Y, a.ylo = ylo, a.R = R, a.rlo = rlo;
  a.c64 = h->coef64, a.c32 = h->coef32, a.cdf = (const df2*)h->coefdf;
  a.wdf = (const df2*)h->wdf, a.w64 = h->w64, a.ws = T.ws;
  a.qmax = h->qcur;
  if (xprec == SG_F32Q && !a.qmax) return sg_fail(h, SG_E_ARG, "apply: grid input without block maxima");
  a.row_ptr = T.row_ptr, a.tj = T.j, a.tk = T.k, a.g64 = T.g, a.g32 = T.gf, a.gdf = (const df2*)T.gdf;
  a.row0 = row0, a.nrows = nrows, a.ybase = ybase, a.rbase = rbase, a.n = h->n, a.m = h->m;
  a.Nx = h->Nx, a.Nc = h->Nc;
  // the mean coupling G_0(i, i) = 1 leads every row of the full and the diagonal tables; with the mean
  // coefficient identically 1 its weight is exactly 1
  a.unit0 = (which == 0 || which == 4) && h->const_mean;
  const int slot = arith == SG_F64 ? 0 : (arith == SG_DF64 ? 2 : 1);
  a.strip = h->apply_strip[slot] > 0 ? h->apply_strip[slot] : STRIP_DEFAULT;
  if (arith == SG_F64) return pick_x<ArF64>(h, a, xprec, yprec, rprec);
  if (arith == SG_DF64) return pick_x<ArDF>(h, a, xprec, yprec, rprec);
  return pick_x<ArF32>(h, a, xprec, yprec, rprec);
}
