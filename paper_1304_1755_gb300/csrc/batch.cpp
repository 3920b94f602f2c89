// Concurrent solves of many independent SG systems of uneven size (grid, M, p).
//
// A small native scheduler: nstreams worker threads, each owning one non-blocking CUDA
// stream, take systems from a shared queue in decreasing order of unknowns (longest job
// first, which bounds the makespan by the largest system plus an even share of the rest)
// and run sg_solve on them.  Every system has its own handle, so its workspace, its
// reduction buffers and its captured preconditioner graphs are private to the worker that
// runs it; the only shared state is the queue index.  While one system's host thread
// waits for a Gram-Schmidt reduction, the other streams keep the GPU busy, which is what
// makes small systems (a few thousand nodes, far below one wave of the GPU) cheap in
// aggregate.
#include <algorithm>
#include <atomic>
#include <numeric>
#include <thread>
#include <vector>

#include "sg_internal.h"

extern "C" int sg_solve_batch(sg_handle* hs, const double* const* F, double* const* U, int nsys,
                              const sg_solve_opts* opts, sg_solve_info* infos, int nstreams) {
  if (!hs || !F || !U || !opts || nsys < 0 || nstreams < 1 || nstreams > 64) return SG_E_ARG;
  for (int s = 0; s < nsys; ++s)
    if (!hs[s] || !F[s] || !U[s]) return SG_E_ARG;
  if (nsys == 0) return SG_OK;
  {
    // a handle's workspace serves one solve at a time: every system needs its own handle
    std::vector<sg_handle> seen(hs, hs + nsys);
    std::sort(seen.begin(), seen.end());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) return SG_E_ARG;
  }
  std::vector<int> order(nsys);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return hs[a]->Nx * (size_t)hs[a]->P > hs[b]->Nx * (size_t)hs[b]->P;
  });
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SG_E_CUDA;
  // every handle must belong to the current device (the worker threads run on it)
  for (int s = 0; s < nsys; ++s)
    if (const int rcd = sg_check_device(hs[s], "sg_solve_batch")) return rcd;
  const int nw = std::min(nstreams, nsys);
  std::vector<cudaStream_t> streams(nw, nullptr);
  for (int w = 0; w < nw; ++w)
    if (cudaStreamCreateWithFlags(&streams[w], cudaStreamNonBlocking) != cudaSuccess) {
      for (int v = 0; v < w; ++v) cudaStreamDestroy(streams[v]);
      return SG_E_CUDA;
    }
  std::atomic<int> next{0};
  std::atomic<int> first_err{SG_OK};
  auto worker = [&](int w) {
    cudaSetDevice(dev);
    for (;;) {
      const int q = next.fetch_add(1);
      if (q >= nsys) break;
      const int s = order[q];
      sg_ctx* h = hs[s];
      cudaStream_t prev = h->stream;
      h->stream = streams[w];
      sg_solve_info info{};
      const int rc = sg_solve(h, F[s], U[s], opts, &info);
      cudaStreamSynchronize(streams[w]);
      h->stream = prev;
      info.status = rc;
      if (infos) infos[s] = info;
      if (rc != SG_OK) {
        int expected = SG_OK;
        first_err.compare_exchange_strong(expected, rc);
      }
    }
  };
  std::vector<std::thread> threads;
  threads.reserve(nw);
  for (int w = 0; w < nw; ++w) threads.emplace_back(worker, w);
  for (auto& t : threads) t.join();
  for (auto s : streams) cudaStreamDestroy(s);
  return first_err.load();
}
