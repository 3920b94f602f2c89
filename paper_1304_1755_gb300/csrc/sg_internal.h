// Internal declarations of the GB300 stochastic Galerkin library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstddef>
#include <cstdint>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "sg.h"

typedef __nv_bfloat16 bf16;

#define SG_MAX_LEVELS 13
// Internal input tag (not in the ABI): an FP32 vector read through its per-PC-block fixed-point grids.
// Block b of the vector (N_x values) has the scale s_b = 2^(148 - e_b), e_b the biased exponent of the
// block's max |z| (block_absmax); a value z stands for its grid value z' = rint(z s_b) / s_b, with
// |z s_b| < 2^22.  The biased integer fma(z, s_b, 1.5 2^23) = 1.5 2^23 + rint(z s_b) is exact in FP32,
// so differences of up to four such values are exact: the double-float operator forms its cell
// features with plain FP32 subtractions.  Blocks with e_b <= 40 (max |z| < 2^-86) read as zero; a
// block with a non-finite value reads as NaN.
#define SG_F32Q 16
#ifdef __CUDACC__
// grid scale / quantum of a block from its max bits (see SG_F32Q); 0 for a block read as zero
// (a non-finite max gives NaN, so a non-finite z_j stays visible to the solver's checks)
__device__ __forceinline__ float qgrid_scale(unsigned maxbits) {
  const int eb = (int)(maxbits >> 23);
  return eb == 255 ? __int_as_float(0x7fc00000) : (eb <= 40 ? 0.f : __int_as_float((148 - eb + 127) << 23));
}
__device__ __forceinline__ float qgrid_quantum(unsigned maxbits) {
  const int eb = (int)(maxbits >> 23);
  return eb == 255 ? __int_as_float(0x7fc00000) : (eb <= 40 ? 0.f : __int_as_float((eb - 148 + 127) << 23));
}
#endif
#define SG_QBIAS 12582912.0f   // 1.5 * 2^23
#define SG_MAX_RESTART 64
#define SG_NTHREADS_RED 256

// Scalar load/store with conversion to the arithmetic type.
template <typename TA, typename TS> __device__ __forceinline__ TA ld_as(const TS* p) { return (TA)(*p); }
template <> __device__ __forceinline__ float ld_as<float, bf16>(const bf16* p) { return __bfloat162float(*p); }
template <> __device__ __forceinline__ double ld_as<double, bf16>(const bf16* p) { return (double)__bfloat162float(*p); }
template <typename TS, typename TA> __device__ __forceinline__ void st_as(TS* p, TA v) { *p = (TS)v; }
template <> __device__ __forceinline__ void st_as<bf16, float>(bf16* p, float v) { *p = __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ void st_as<bf16, double>(bf16* p, double v) { *p = __float2bfloat16_rn((float)v); }

// PC-coupling table in CSR form over rows: for row i the terms t in
// [row_ptr[i], row_ptr[i+1]) contribute  g[t] * K_{k[t]} X_{j[t]}  to Y_i.
struct TermTable {
  int* row_ptr = nullptr;
  int* j = nullptr;
  int* k = nullptr;
  double* g = nullptr;
  float* gf = nullptr;
  float* gdf = nullptr;       // g as double-float pairs (hi, lo)
  int* ws = nullptr;          // weight slot: 0 for the mean term, 1 + (k-1) p + n for c_k gamma(n)
  int nnz = 0;
};

// One multigrid level: vertex count n_l, interior side m_l = n_l - 2.
struct MGLevel {
  int n = 0, m = 0;
  size_t N = 0;               // m * m
  double* st64 = nullptr;     // 9 * N Galerkin stencil (only when the mean is not constant 1)
  float* st32 = nullptr;
};

// Per-storage-precision multigrid and sweep buffers.
struct PrecWork {
  bool ready = false;
  void* T = nullptr;                    // stage right-hand side, n_q_max * N_x
  void* T32 = nullptr;                  // FP32 stage right-hand side (SG_BF16Z sweeps), n_q_max * N_x
  void* b[SG_MAX_LEVELS] = {};          // level >= 1 right-hand sides, P * N_l
  void* x[SG_MAX_LEVELS] = {};          // level >= 1 solutions, P * N_l
  void* S1 = nullptr;                   // symmetric sweep: lower-sweep result (P * N_x)
  void* S2 = nullptr;                   //                  K_0 times it, FP32 (FP64 for an FP64 sweep)
  int s1_prec = -1;                     // storage precision of S1
};

// Per-phase event tracing (sg_timing_*).  Phase 0 outer operator, 1 preconditioner,
// 2 Gram-Schmidt, 3 other.
struct Tracer {
  bool on = false;
  struct Span { cudaEvent_t a, b; int phase; };
  std::vector<cudaEvent_t> pool;
  std::vector<Span> spans;
  long long launches[4] = {0, 0, 0, 0};
};

struct sg_ctx {
  // problem
  int n = 0, m = 0, M = 0, p = 0, P = 0, family = 0;
  size_t Nx = 0, Nc = 0;
  size_t Np = 0;                        // P * Nx rounded up to a multiple of 64 (Krylov vector stride)
  int nu1 = 1, nu2 = 1;
  double omega = 8.0 / 9.0;
  bool const_mean = true;
  int elements = SG_Q1;                 // SG_Q1 or SG_P1 (the paper's triangles, point Gauss-Seidel cycle)
  int gs_order = SG_GS_LEX;             // SG_P1 smoother order (lexicographic or red-black)
  // B_T applications with FP32 output may also record their output's per-block maxima (the grid scales
  // of the flexible basis) in the level-0 multigrid kernels: the caller sets zmax_out, the sweep sets
  // zmax_done when it did so
  unsigned* zmax_out = nullptr;
  bool zmax_done = false;
  double* bsr = nullptr;                // recursive B_S: per depth q >= 1 a copy of the blocks of degree < q
  size_t bsr_off[12] = {};              // (p <= 10)
  double* ew = nullptr;                 // SG_P1: edge weights per mode, (M+1) x 2 x n^2 (horizontal, vertical)
  double* p1w = nullptr;                // SG_P1: V-cycle workspace, P x p1w_ld doubles
  size_t p1w_ld = 0;
  int device = -1;                      // the CUDA device the handle was set up on
  cudaStream_t stream = nullptr;
  std::vector<int> alpha;               // P * M
  std::vector<int> lvl_off;             // p + 2 offsets of the degree levels
  std::vector<double> coef_h;           // (M+1) * Nc
  // device operator data
  double* coef64 = nullptr;             // (M+1) * Nc
  float* coef32 = nullptr;
  float* coefdf = nullptr;              // (M+1) * Nc double-float pairs (hi, lo)
  float* wdf = nullptr;                 // (1 + M p) * Nc double-float weights c_k(e) gamma(n) (or null)
  double* w64 = nullptr;                // the same weights in FP64 (or null)
  TermTable t_all, t_lower, t_upper, t_off, t_diag;   // all / lower / upper / off-diagonal / mean term
  double* pvec = nullptr;               // P doubles of device scratch (objective)
  unsigned* qmax = nullptr;             // (SG_MAX_RESTART + 1) x P block maxima (float bits) of the z_j (SG_F32Q)
  const unsigned* qcur = nullptr;       // the maxima of the SG_F32Q input of the next launch_apply
  // exact lower-degree block (SG_PC_BLOCKTRI_EXACT): the degree-(p-1) handle and its inner solve settings
  sg_ctx* child = nullptr;
  double inner_tol = 1e-12;
  int inner_restart = 30;
  double* xbuf = nullptr;               // P * Nx doubles (right-hand side of the transposed inner solve)
  // multigrid hierarchy
  int nlev = 0;
  int lc = 0;                           // first level handled by the single-CTA coarse kernel
  MGLevel lev[SG_MAX_LEVELS];
  PrecWork work[3];
  // Krylov workspace (allocated on first solve)
  double* red_partial = nullptr;        // reduction partials
  double* red_out = nullptr;            // reduction results (device)
  unsigned* red_count = nullptr;
  double* red_host = nullptr;           // pinned
  int red_blocks = 0;
  double* kv = nullptr;                 // (restart + 1) FP64 vectors
  int kv_cap = 0;
  int kv_layout = -1;                   // 0: FP64 basis vectors, 1: double-float (what the padding holds)
  void* kz = nullptr;                   // restart vectors in pc precision
  int kz_cap = 0, kz_prec = -1;
  double* ktmp = nullptr;               // 4 FP64 work vectors
  double* dstage = nullptr;             // staging for host F/U (2 vectors)
  Tracer tr;
  int phase = 3;
  bool true_res_valid = false;          // the solver already computed the final FP64 true residual
  // Host-buffer solves: the iterate is copied to the caller's U on a side stream while its true
  // residual is being checked, since the check usually confirms convergence.
  double* spec_dst = nullptr;           // host destination of U (null: no early copy)
  cudaStream_t cstream = nullptr;       // side stream of the early copy
  cudaEvent_t ev_u = nullptr, ev_c = nullptr;   // U ready / copy done
  bool spec_pending = false;            // an early copy was issued and U has not changed since
  int apply_strip[3] = {0, 0, 0};       // operator kernel strip height per arithmetic (FP64, FP32, DF); 0 = default
  // CUDA graphs of whole preconditioner applications, keyed by their operands
  struct GraphEntry {
    cudaGraphExec_t exec;
    long long kernels;
  };
  std::map<std::tuple<const void*, const void*, int, int, int, const void*>, GraphEntry> graphs;
  std::string err;
};

inline void count_launch(sg_ctx* h, int k = 1) { h->tr.launches[h->phase] += k; }

// Sets the current phase and, when tracing, brackets the enclosed launches with events.
struct PhaseScope {
  sg_ctx* h;
  int prev;
  cudaEvent_t b = nullptr;
  PhaseScope(sg_ctx* h_, int ph) : h(h_), prev(h_->phase) {
    h->phase = ph;
    if (h->tr.on) {
      cudaEvent_t a = take_event(h);
      b = take_event(h);
      cudaEventRecord(a, h->stream);
      h->tr.spans.push_back({a, b, ph});
    }
  }
  ~PhaseScope() {
    if (b) cudaEventRecord(b, h->stream);
    h->phase = prev;
  }
  static cudaEvent_t take_event(sg_ctx* h) {
    if (h->tr.pool.empty()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      return e;
    }
    cudaEvent_t e = h->tr.pool.back();
    h->tr.pool.pop_back();
    return e;
  }
};

// error helpers
int sg_fail(sg_ctx* h, int code, const std::string& msg);
// SG_OK when the calling thread's current device is the handle's, else SG_E_STATE (nothing launched)
int sg_check_device(sg_ctx* h, const char* who);
#define SG_CUDA(h, call)                                                          \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess)                                                        \
      return sg_fail((h), SG_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

size_t prec_size(int prec);
// Preconditioner modes: the storage precision of the returned vectors Z and of the work
// buffers (levels, stage right-hand sides).  Only SG_BF16Z differs: BF16 work, FP32 Z.
inline int zprec_of(int mode) { return mode == SG_BF16Z ? SG_F32 : mode; }
inline int wprec_of(int mode) { return mode == SG_BF16Z ? SG_BF16 : mode; }

// setup.cpp
int kl_coef_host(int n, int M, double sigma, double corr_len, const double* abar, double* coef, double* lam);
int kl_coef_p1_host(int n, int M, double sigma, double corr_len, double* coef, double* lam);
void build_basis(int M, int p, std::vector<int>& alpha, std::vector<int>& lvl_off);
double gamma_1d(int family, int nn);
void build_terms(const sg_ctx* h, int which, std::vector<int>& row_ptr, std::vector<int>& tj,
                 std::vector<int>& tk, std::vector<double>& tg);
void galerkin_stencils(int n0, int nlev, const double* abar_cells, std::vector<std::vector<double>>& st);

// api.cu: the preconditioner dispatch and the Krylov workspace of sg_solve (layout 0: FP64 basis)
int apply_precond_ext(sg_ctx* h, int pc, int rprec, const void* R, void* Z, int prec, int transpose);
int ensure_krylov_ext(sg_ctx* h, int nv, int nz, int zprec, int layout);

// k_apply.cu
// which: 0 = all terms (Y = A X), 1 = lower terms, 2 = upper terms, 3 = off-diagonal terms,
// 4 = the mean term only (Y = (I (x) K_0) X).
// Computes Y_i (i in [row0, row0 + nrows)) = epi ? R_i - S_i : S_i,
// S_i = sum over the table's terms; Y rows are offset by ybase, R rows by rbase.
// Precisions: SG_F64 / SG_F32 / SG_BF16 plain arrays, SG_DF64 hi array with the lo
// array at offset *lo (elements).  arith: SG_F64, SG_F32 or SG_DF64.
int launch_apply(sg_ctx* h, int which, int xprec, const void* X, size_t xlo, int yprec, void* Y, size_t ylo,
                 int rprec, const void* R, size_t rlo, int row0, int nrows, int ybase, int rbase, int arith);

// k_p1.cu (SG_P1 handles): the operator (FP64; same arguments as launch_apply) and the point
// Gauss-Seidel V-cycle (FP64 B with leading dimension ldb, FP64 X with ldx)
int launch_apply_p1(sg_ctx* h, int which, int xprec, const void* X, int yprec, void* Y, int rprec, const void* R,
                    int row0, int nrows, int ybase, int rbase, int arith);
int vcycle_p1(sg_ctx* h, int nb, const double* B, size_t ldb, double* X, size_t ldx);
int setup_p1(sg_ctx* h);

// k_mg.cu
// bguard: B lies in a guarded buffer (sg_galloc), so the tile loaders may over-fetch around it
int vcycle_run(sg_ctx* h, int prec, int nb, const void* B, int bprec, void* X, bool bguard = false,
               unsigned* zmax = nullptr);
// device buffers with 256 bytes before and 4 KB after the data, for the multigrid tile loaders
void* sg_galloc(size_t bytes);
void sg_gfree(void* p);
int ensure_prec_work(sg_ctx* h, int prec);
// R is FP64 (rprec SG_F64) or FP32 (rprec SG_F32, e.g. the hi array of a double-float vector)
int precond_blocktri(sg_ctx* h, int rprec, const void* R, void* Z, int prec, int transpose);
int precond_blockdiag(sg_ctx* h, int rprec, const void* R, void* Z, int prec);
int precond_blocksym(sg_ctx* h, int rprec, const void* R, void* Z, int prec);
int precond_blocksym_rec(sg_ctx* h, int rprec, const void* R, void* Z, int prec);

// k_vec.cu
int vec_dots(sg_ctx* h, const double* V, size_t ldv, int nv, const double* w, size_t N, bool with_ww, double* out_host);
int vec_axpys_norm(sg_ctx* h, const double* V, size_t ldv, int nv, const double* hcoef_dev, double* w, size_t N,
                   double* nrm2_host);
int vec_update(sg_ctx* h, double* U, int zprec, const void* Z, size_t ldz, int nz, const double* y_host, size_t N);
int vec_cast(sg_ctx* h, int iprec, const void* in, int oprec, void* out, size_t N);
int vec_axpby(sg_ctx* h, double a, const double* x, double b, double* y, size_t N);   // y = a x + b y
int vec_fill(sg_ctx* h, double* y, size_t N, double v);    // by a kernel (also for mapped host memory)
// F = e_0 (x) (w f): F[s] = w f[s] (w f when f is null) for s < Nx, zero for the other PC blocks
int vec_load(sg_ctx* h, const double* f, double w, double* F);
// qmax[b] = bits of max |Z| over block b (P blocks of N_x consecutive values): the grids of SG_F32Q
int block_absmax(sg_ctx* h, const float* Z, unsigned* qmax);
// U += sum_l y_l z'_l with z'_l the grid values (SG_F32Q) of the FP32 z_l, block maxima qmax + l P;
// FP64 U (vec_update_q) or double-float U with the lo array at + lo (df_update_q)
int vec_update_q(sg_ctx* h, double* U, const float* Z, size_t ldz, int nz, const double* y_host, size_t N,
                 const unsigned* qmax);
int df_update_q(sg_ctx* h, float* U, size_t lo, const float* Z, size_t ldz, int nz, const double* y_host, size_t N,
                const unsigned* qmax);
int vec_dot_pairs(sg_ctx* h, int npairs, const double* const* xs, const void* const* ys, const int* yprecs,
                  size_t N, double* out_host);
int vec_axpy_prec(sg_ctx* h, double a, int xprec, const void* x, double* y, size_t N);  // y += a x
int ensure_reduction(sg_ctx* h);
int copy_red(sg_ctx* h, int slot, int count, double* out_host);
// host -> reduction slot (device), stream-ordered; slot 3 carries Gram-Schmidt coefficients
int upload_red(sg_ctx* h, int slot, const double* host, int count);
const double* red_slot(const sg_ctx* h, int slot);
// Double-float Krylov vectors: hi[0..Np), lo[Np..2Np) with the padded length Np (a multiple
// of 64, padding kept at zero); dots/axpys/scale take Np, the others the true length N
// and the lo offset.
int df_dots(sg_ctx* h, const float* V, size_t ldv, int nv, const float* w, size_t Np, bool with_ww);   // red slot 0
int df_axpys_norm(sg_ctx* h, const float* V, size_t ldv, int nv, const double* hc_dev, float* w, size_t Np);  // slot 1
int df_update(sg_ctx* h, float* U, size_t lo, int zprec, const void* Z, size_t ldz, int nz, const double* y_host,
              size_t N);
int df_from_f64(sg_ctx* h, const double* x, float* y, size_t N, size_t lo);
int df_to_f64(sg_ctx* h, const float* x, double* y, size_t N, size_t lo);
// adjoint helpers
int adj_cell_forms(sg_ctx* h, const double* U, const double* L, double* g_abar);
int objective_dots(sg_ctx* h, const double* U, double* mu_host);
int objective_grad(sg_ctx* h, const double* mu_dev, double* G);
