// Batched form: many contours of uneven size solved for the same plane waves.
//
// The paper's solver serves any number of right-hand sides for one contour
// (Sec. V, Eq. 9); a batch adds the other axis, many contours.  Their stored
// operators do not fit together (64 star contours with N up to 16384 hold
// ~565 GB of split-bf16 planes), so contours stream through a fixed number of
// contexts: `workers` host threads, each owning one context on its own CUDA
// stream, take contours from a queue ordered by decreasing N (the longest
// start first, the short ones fill in at the end) and run mesh, assembly,
// skeleton, factor and the plane-wave solve on their stream.  The streams
// overlap one contour's setup with another's solve on the GPU, and a
// context's buffers are reused by its next contour.  Every per-run table the
// kernels read is passed by value, so contexts of different contours assemble
// at the same time safely.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <string>
#include <thread>
#include <vector>

#include "../../include/wcs.h"
#include "internal.h"

using namespace wcs;

extern "C" int wcs_batch_solve_fourier(const wcs_options* opt, int count, int nf, const double* cos_c,
                                       const double* sin_c, const int64_t* N, const double* k, int64_t B,
                                       const double* angles_host, double tol, int rank_div, uint64_t seed,
                                       int workers, double* j_host, wcs_batch_stats* stats) {
  if (count < 0 || nf < 1 || nf > 64 || (count > 0 && (!cos_c || !N || !k || !j_host)) || B < 0 ||
      (B > 0 && !angles_host) || !(tol >= 0) || workers < 1 || workers > 8) {
    set_error("batch: bad argument (count >= 0, 1 <= nf <= 64, pointers, 1 <= workers <= 8)");
    return WCS_ERR_ARG;
  }
  for (int c = 0; c < count; ++c)
    if (N[c] < 12 || !(cos_c[(int64_t)c * nf] > 0)) {
      set_error("batch: contour " + std::to_string(c) + " has N < 12 or a non-positive mean radius");
      return WCS_ERR_ARG;
    }
  if (count == 0 || B == 0) return WCS_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { set_error("batch: no current device"); return WCS_ERR_CUDA; }
  std::vector<int> order(count);
  for (int c = 0; c < count; ++c) order[c] = c;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return N[a] > N[b]; });
  std::vector<int64_t> off(count + 1, 0);
  for (int c = 0; c < count; ++c) off[c + 1] = off[c] + 2 * N[c] * B;   // doubles
  std::vector<wcs_batch_stats> st(count);
  std::atomic<int> next{0};
  std::vector<std::string> errs(count);
  const int nw = std::min(workers, count);
  auto work = [&](int w) {
    cudaSetDevice(dev);
    cudaStream_t s = nullptr;
    wcs_ctx* ctx = nullptr;
    int boot = (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess) ? WCS_OK : WCS_ERR_CUDA;
    if (!boot) boot = wcs_create(&ctx, opt, (void*)s);
    for (;;) {
      const int i = next.fetch_add(1);
      if (i >= count) break;
      const int c = order[i];
      wcs_batch_stats& r = st[c];
      r = wcs_batch_stats{};
      r.worker = w;
      r.rank = -1;
      if (boot) { r.status = boot; errs[c] = "worker set-up failed"; continue; }
      const auto t0 = std::chrono::steady_clock::now();
      int rc = wcs_contour_fourier(ctx, nf, cos_c + (int64_t)c * nf, sin_c ? sin_c + (int64_t)c * nf : nullptr);
      if (!rc) rc = wcs_mesh(ctx, N[c], k[c]);
      if (!rc) rc = wcs_assemble(ctx);
      int rank = 0;
      if (!rc) {
        const int cap = rank_div > 0 ? (int)std::max<int64_t>(1, N[c] / rank_div) : 0;
        rc = wcs_skeleton(ctx, tol, cap, seed, &rank);
        if (rc == WCS_ERR_RANK_CAP) rc = WCS_OK;
      }
      if (!rc) rc = wcs_factor(ctx);
      const auto t1 = std::chrono::steady_clock::now();
      wcs_solve_info si{};
      if (!rc) rc = wcs_solve_planewaves_host(ctx, B, angles_host, j_host + off[c], N[c], &si);
      const auto t2 = std::chrono::steady_clock::now();
      r.status = rc;
      r.rank = rank;
      r.refine_steps = si.refine_steps;
      r.rel_residual = si.rel_residual;
      r.setup_s = std::chrono::duration<double>(t1 - t0).count();
      r.solve_s = std::chrono::duration<double>(t2 - t1).count();
      if (rc && rc != WCS_ERR_NOT_CONVERGED) errs[c] = wcs_last_error();
    }
    if (ctx) wcs_destroy(ctx);
    if (s) cudaStreamDestroy(s);
  };
  std::vector<std::thread> th;
  for (int w = 0; w < nw; ++w) th.emplace_back(work, w);
  for (auto& t : th) t.join();
  int status = WCS_OK;
  for (int c = 0; c < count; ++c) {
    if (stats) stats[c] = st[c];
    if (st[c].status && st[c].status != WCS_ERR_NOT_CONVERGED && (status == WCS_OK || status == WCS_ERR_NOT_CONVERGED)) {
      status = st[c].status;
      set_error("batch: contour " + std::to_string(c) + ": " + errs[c]);
    } else if (st[c].status == WCS_ERR_NOT_CONVERGED && status == WCS_OK) {
      status = WCS_ERR_NOT_CONVERGED;
      set_error("batch: contour " + std::to_string(c) + " did not reach refine_tol");
    }
  }
  return status;
}
