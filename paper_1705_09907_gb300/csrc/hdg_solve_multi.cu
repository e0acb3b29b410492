// Several independent problems of uneven size solved together (the uneven
// instances of hdg_setup_batch): each context's multigrid-preconditioned CG
// runs on a stream of its own, issued from a host thread of its own, so the
// instances' kernels and captured V-cycle graphs share the GPU at the same time
// -- a small mesh fills the SMs a large one leaves idle instead of waiting for
// it. Every instance runs exactly the kernels of its own hdg_solve, so each
// result is bitwise that of the instance solved alone.
#include <thread>
#include <vector>

#include "hdg_internal.h"

using namespace hdg;

extern "C" int hdg_solve_multi(int n, void* const* ctxs, const double* const* b, double* const* lambda,
                               double rtol, int maxit, int inner, hdg_solve_info* infos, int* statuses,
                               void* stream) {
  if (n < 1 || n > 64 || !ctxs || !b || !lambda || !(rtol > 0.0) || maxit < 1) return HDG_ERR_INVALID_ARG;
  if (inner < 0 || inner > 3) return HDG_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HDG_ERR_CUDA;
  for (int q = 0; q < n; ++q) {
    Context* c = (Context*)ctxs[q];
    if (!c || !b[q] || !lambda[q] || b[q] == lambda[q]) return HDG_ERR_INVALID_ARG;
    if (c->dev != dev) return HDG_ERR_INVALID_ARG;
    if (inner != HDG_PREC_FP64 && !c->opt.mixed) return HDG_ERR_UNSUPPORTED;
    for (int r = 0; r < q; ++r)
      if (ctxs[r] == ctxs[q]) return HDG_ERR_INVALID_ARG;    // one context, one solve at a time
  }
  cudaStream_t caller = (cudaStream_t)stream;
  std::vector<cudaStream_t> st(n, nullptr);
  std::vector<cudaEvent_t> done(n, nullptr);
  cudaEvent_t start = nullptr;
  int status = HDG_OK;
  auto fail = [&](int code) { if (status == HDG_OK) status = code; };
  if (cudaEventCreateWithFlags(&start, cudaEventDisableTiming) != cudaSuccess) return HDG_ERR_CUDA;
  if (cudaEventRecord(start, caller) != cudaSuccess) fail(HDG_ERR_CUDA);
  for (int q = 0; q < n && status == HDG_OK; ++q) {
    if (cudaStreamCreateWithFlags(&st[q], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&done[q], cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamWaitEvent(st[q], start, 0) != cudaSuccess)   // after the caller's earlier work
      fail(HDG_ERR_CUDA);
  }
  std::vector<int> res(n, HDG_ERR_CUDA);
  if (status == HDG_OK) {
    std::vector<std::thread> th;
    th.reserve(n);
    for (int q = 0; q < n; ++q) {
      th.emplace_back([&, q]() {
        if (cudaSetDevice(dev) != cudaSuccess) return;
        hdg_solve_info* inf = infos ? &infos[q] : nullptr;
        res[q] = hdg_solve(ctxs[q], b[q], lambda[q], 1, rtol, maxit, inner, inf, st[q]);
        cudaEventRecord(done[q], st[q]);
      });
    }
    for (auto& t : th) t.join();
    for (int q = 0; q < n; ++q) {
      if (statuses) statuses[q] = res[q];
      if (res[q] != HDG_OK) fail(res[q]);
      if (cudaStreamWaitEvent(caller, done[q], 0) != cudaSuccess) fail(HDG_ERR_CUDA);
    }
  }
  for (int q = 0; q < n; ++q) {
    if (st[q]) { cudaStreamSynchronize(st[q]); cudaStreamDestroy(st[q]); }
    if (done[q]) cudaEventDestroy(done[q]);
  }
  cudaEventDestroy(start);
  return status;
}
