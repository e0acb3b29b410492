// Several independent problems of uneven size solved together (the uneven
// instances of hdg_setup_batch). With CUDA graphs on in every context (and no
// FMG start) all instances are one graph and one launch: per instance a chain
// prologue -> conditional WHILE node running that context's CG iterations
// (the device-resident loop of hdg_solve) -> copy of the solution; the chains
// are independent, so the GPU runs them side by side -- a small mesh fills the
// SMs a large one leaves idle -- and the host waits once. Otherwise each
// context's solve runs on a stream of its own, issued from a host thread of its
// own. Either way every instance runs exactly the kernels of its own hdg_solve,
// so each result is bitwise that of the instance solved alone.
#include <chrono>
#include <thread>
#include <vector>

#include "hdg_internal.h"

using namespace hdg;

static int map_err(cudaError_t e) { return e == cudaErrorMemoryAllocation ? HDG_ERR_OOM : HDG_ERR_CUDA; }

// All instances in one graph (see the file comment); HDG_ERR_UNSUPPORTED when the
// graph cannot be built (no conditional nodes), before anything was launched.
static int solve_multi_graph(int n, void* const* ctxs, const double* const* b, double* const* lambda, double rtol,
                             int maxit, int inner, hdg_solve_info* infos, int* statuses, cudaStream_t s) {
  cudaGraph_t G = nullptr;
  cudaStream_t cs = nullptr;
  cudaGraphExec_t ge = nullptr;
  if (cudaGraphCreate(&G, 0) != cudaSuccess) return HDG_ERR_CUDA;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  for (int q = 0; q < n && e == cudaSuccess; ++q)
    e = cg_multi_add((Context*)ctxs[q], inner, b[q], lambda[q], rtol, maxit, G, cs);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, G, 0);
  cudaGraphDestroy(G);
  if (cs) cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return HDG_ERR_UNSUPPORTED;
  }
  const auto t0 = std::chrono::steady_clock::now();
  e = cudaGraphLaunch(ge, s);
  for (int q = 0; q < n && e == cudaSuccess; ++q) e = cg_multi_fetch((Context*)ctxs[q], s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaGraphExecDestroy(ge);
  if (e != cudaSuccess) return map_err(e);
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  int status = HDG_OK;
  for (int q = 0; q < n; ++q) {
    Context* c = (Context*)ctxs[q];
    hdg_solve_info* inf = infos ? &infos[q] : nullptr;
    int r = cg_multi_result(c, inf);
    // a bounded wait that gave up inside an apply (the context's error flag)
    int h = 0;
    if (cudaMemcpy(&h, c->err_flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) r = HDG_ERR_CUDA;
    if (h != 0) {
      cudaMemset(c->err_flag, 0, sizeof(int));
      if (r == HDG_OK || r == HDG_ERR_NOT_CONVERGED || r == HDG_ERR_BREAKDOWN)
        r = h == 2 ? HDG_ERR_TIMEOUT : (h == 1 || h == 3) ? HDG_ERR_INVALID_ARG : HDG_ERR_CUDA;
    }
    if (inf) inf->solve_ms = ms;
    if (statuses) statuses[q] = r;
    if (r != HDG_OK && status == HDG_OK) status = r;
  }
  return status;
}

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
  bool one_graph = true;
  for (int q = 0; q < n; ++q) {
    const Context* c = (const Context*)ctxs[q];
    one_graph = one_graph && c->opt.use_graphs && !c->opt.fmg_start && c->cg_x && c->h_cg && !c->cg_graph_failed;
  }
  if (one_graph) {
    const int st = solve_multi_graph(n, ctxs, b, lambda, rtol, maxit, inner, infos, statuses, caller);
    if (st != HDG_ERR_UNSUPPORTED) return st;   // else: conditional graphs unavailable, use the threads
  }
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
