// Tile autotuner for the operator kernel (k_apply).
//
// The kernel's tile is a warp column of 31 cells times a strip of node rows; the strip
// height trades the one primer cell row per strip (short strips) against the number of
// warps available to cover the grid (tall strips leave small grids with too few warps).
// The best height depends on the grid, the number of PC rows and the arithmetic, so it is
// measured: every candidate is timed with CUDA events on the handle's stream for the
// full operator (all couplings) in the three arithmetic forms the solvers use, and the
// fastest is kept in the handle.  Results are cached for the process by problem shape,
// so a batch of many systems of few distinct sizes tunes each size once.
#include <array>
#include <map>
#include <mutex>
#include <tuple>

#include "sg_internal.h"

namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, bool>, std::array<int, 3>> g_tuned;   // (n, M, p, nnz, const mean)
constexpr int kStrips[] = {4, 8, 16, 32, 64};
}  // namespace

extern "C" int sg_autotune(sg_handle h, int which) {
  if (!h) return SG_E_ARG;
  if (const int rcd = sg_check_device(h, "sg_autotune")) return rcd;
  if (h->elements != SG_Q1) return SG_OK;                 // the P1 operator has no tile to tune
  if (which == 0) which = 7;
  const auto key = std::make_tuple(h->n, h->M, h->p, h->t_all.nnz, h->const_mean);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tuned.find(key);
  if (it != g_tuned.end()) {
    for (int s = 0; s < 3; ++s)
      if (which & (1 << s)) h->apply_strip[s] = it->second[s];
    return SG_OK;
  }
  const size_t N = h->Nx * (size_t)h->P;
  void *X = nullptr, *Y = nullptr;
  if (cudaMalloc(&X, sizeof(double) * N) != cudaSuccess) return sg_fail(h, SG_E_ALLOC, "autotune: buffers");
  if (cudaMalloc(&Y, sizeof(double) * N) != cudaSuccess) {
    cudaFree(X);
    return sg_fail(h, SG_E_ALLOC, "autotune: buffers");
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int rc = SG_OK;
  std::array<int, 3> best{0, 0, 0};
  if (cudaMemsetAsync(X, 0, sizeof(double) * N, h->stream) != cudaSuccess) rc = sg_fail(h, SG_E_CUDA, "autotune: memset");
  // slot 0: FP64 arithmetic on FP64 vectors; 1: FP32 on BF16 in/out; 2: double-float, BF16 in, DF out
  const int arith[3] = {SG_F64, SG_F32, SG_DF64};
  const int xp[3] = {SG_F64, SG_BF16, SG_BF16};
  const int yp[3] = {SG_F64, SG_BF16, SG_DF64};
  for (int s = 0; s < 3 && rc == SG_OK; ++s) {
    if (!(which & (1 << s))) continue;
    float tbest = 1e30f;
    for (int strip : kStrips) {
      h->apply_strip[s] = strip;
      for (int rep = 0; rep < 4 && rc == SG_OK; ++rep) {     // one warm-up, three timed
        if (rep == 1) cudaEventRecord(e0, h->stream);
        rc = launch_apply(h, 0, xp[s], X, 0, yp[s], Y, N, SG_F64, nullptr, 0, 0, h->P, 0, 0, arith[s]);
      }
      if (rc) break;
      cudaEventRecord(e1, h->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        rc = sg_fail(h, SG_E_CUDA, "autotune: timing");
        break;
      }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < tbest) tbest = ms, best[s] = strip;
    }
    h->apply_strip[s] = best[s];
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(X);
  cudaFree(Y);
  if (rc == SG_OK && which == 7) g_tuned.emplace(key, best);
  return rc;
}
