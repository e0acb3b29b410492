// C ABI entry points (declared in include/hdg.h).
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "hdg_internal.h"

namespace hdg {
cudaError_t launch_maps(Context* c, cudaStream_t s);
cudaError_t launch_check_kappa(Context* c, cudaStream_t s);
}  // namespace hdg

using namespace hdg;

static int map_cuda(cudaError_t e) {
  if (e == cudaSuccess) return HDG_OK;
  if (e == cudaErrorMemoryAllocation) return HDG_ERR_OOM;
  if (e == cudaErrorInvalidValue) return HDG_ERR_INVALID_ARG;
  return HDG_ERR_CUDA;
}

#define TRY(expr)                                  \
  do {                                             \
    cudaError_t _e = (expr);                       \
    if (_e != cudaSuccess) return map_cuda(_e);    \
  } while (0)

// Reads and clears the device error flag (synchronises the stream).
static int read_err_flag(Context* c, cudaStream_t s) {
  int h = 0;
  TRY(cudaMemcpyAsync(&h, c->err_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));
  if (h != 0) {
    TRY(cudaMemsetAsync(c->err_flag, 0, sizeof(int), s));
    TRY(cudaStreamSynchronize(s));
  }
  switch (h) {
    case 0: return HDG_OK;
    case 2: return HDG_ERR_TIMEOUT;
    case 1: case 3: return HDG_ERR_INVALID_ARG;   // non-SPD local system / bad kappa
    default: return HDG_ERR_CUDA;
  }
}

extern "C" {

void hdg_default_options(hdg_options* o) {
  if (!o) return;
  o->nu1 = 2; o->nu2 = 2; o->coarse_n = 2; o->tau = 1.0; o->cheb_degree = 2; o->mixed = 1; o->use_graphs = 1;
  o->autotune = 1; o->reduced = 1; o->tau_kappa = 0;
  o->smoother = 0; o->tensor_apply = 1; o->fmg_start = 0; o->max_device_bytes = 0; o->wait_probe = 0;
  o->coarse_fuse = 1; o->top_accum = 1;
}

const char* hdg_error_string(int s) {
  switch (s) {
    case HDG_OK: return "ok";
    case HDG_ERR_INVALID_ARG: return "invalid argument";
    case HDG_ERR_CUDA: return "CUDA error";
    case HDG_ERR_OOM: return "out of device memory";
    case HDG_ERR_NOT_CONVERGED: return "not converged within the iteration limit";
    case HDG_ERR_BREAKDOWN: return "CG breakdown (p^T A p <= 0 or not finite)";
    case HDG_ERR_TIMEOUT: return "a bounded device wait gave up";
    case HDG_ERR_UNSUPPORTED: return "unsupported request";
    default: return "unknown status";
  }
}

static int setup_impl(Context* c, const double* kappa, cudaStream_t s) {
  const int k = c->k;
  TRY(cudaGetDevice(&c->dev));
  TRY(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->dev));
  TRY(cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->dev));
  build_ref_tables(k, c->hx, c->hy, c->ref);
  // upload the finest tables in one buffer
  std::vector<double> pack;
  auto put = [&](const std::vector<double>& v) { size_t o = pack.size(); pack.insert(pack.end(), v.begin(), v.end()); return o; };
  c->off_P = put(c->ref.P); c->off_Mb = put(c->ref.Mb); c->off_Z = put(c->ref.Z); c->off_Eb = put(c->ref.Eb);
  c->off_Y = put(c->ref.Y); c->off_Ml = put(c->ref.Ml); c->off_MiBt = put(c->ref.MiBt); c->off_MiC = put(c->ref.MiC);
  c->off_Vf = put(c->ref.Vf); c->off_wJf = put(c->ref.wJf); c->off_M = put(c->ref.M);
  // transposed copies: the warp-per-element kernels read a matrix's column
  // (one entry per lane) as one contiguous row of the transpose
  {
    const RefTables& r = c->ref;
    auto tr = [](const double* a, int rows, int cols) {
      std::vector<double> t((size_t)rows * cols);
      for (int i = 0; i < rows; ++i)
        for (int j = 0; j < cols; ++j) t[(size_t)j * rows + i] = a[(size_t)i * cols + j];
      return t;
    };
    c->off_ZT = put(tr(r.Z.data(), r.n, r.m));
    c->off_EbT = put(tr(r.Eb.data(), r.n, r.m));
    std::vector<double> mibt, mic;
    for (int cmp = 0; cmp < 2; ++cmp) {
      const std::vector<double> a = tr(r.MiBt.data() + (size_t)cmp * r.n * r.n, r.n, r.n);
      const std::vector<double> b = tr(r.MiC.data() + (size_t)cmp * r.n * r.m, r.n, r.m);
      mibt.insert(mibt.end(), a.begin(), a.end());
      mic.insert(mic.end(), b.begin(), b.end());
    }
    c->off_MiBtT = put(mibt);
    c->off_MiCT = put(mic);
    c->off_VfT = put(tr(r.Vf.data(), r.nf, r.n));
  }
  {
    // postprocessing tables, transposed so that lane o reads entry o of a row
    std::vector<double> Hq, mu, Dn;
    build_post_tables(k, c->hx, c->hy, Hq, mu, Dn);
    const int n = c->ref.n, ns = (k + 2) * (k + 2);
    c->post_ns = ns;
    std::vector<double> post((size_t)2 * n * ns + n + (size_t)2 * ns * ns);
    for (int cmp = 0; cmp < 2; ++cmp)
      for (int i = 0; i < ns; ++i)
        for (int j = 0; j < n; ++j) post[(size_t)cmp * n * ns + (size_t)j * ns + i] = Hq[(size_t)cmp * ns * n + i * n + j];
    for (int j = 0; j < n; ++j) post[(size_t)2 * n * ns + j] = mu[j];
    double* dn = post.data() + (size_t)2 * n * ns + n;
    for (int cmp = 0; cmp < 2; ++cmp)
      for (int i = 0; i < ns; ++i)
        for (int kk = 0; kk < ns; ++kk) dn[(size_t)cmp * ns * ns + (size_t)kk * ns + i] = Dn[(size_t)cmp * ns * ns + i * ns + kk];
    TRY(ctx_alloc(c, (void**)&c->d_post, post.size() * sizeof(double)));
    TRY(cudaMemcpyAsync(c->d_post, post.data(), post.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    TRY(cudaStreamSynchronize(s));   // the host vector goes out of scope
  }
  TRY(ctx_alloc(c, (void**)&c->d_ref, pack.size() * sizeof(double)));
  TRY(cudaMemcpyAsync(c->d_ref, pack.data(), pack.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  // [0]: error flag; [1]: launches left that test the bounded-wait path
  TRY(ctx_alloc(c, (void**)&c->err_flag, 2 * sizeof(int)));
  TRY(cudaMemsetAsync(c->err_flag, 0, 2 * sizeof(int), s));
  TRY(ctx_alloc(c, (void**)&c->kappa, (size_t)c->nel * sizeof(double)));
  TRY(cudaMemcpyAsync(c->kappa, kappa, (size_t)c->nel * sizeof(double), cudaMemcpyDeviceToDevice, s));
  TRY(launch_check_kappa(c, s));
  {
    int st = read_err_flag(c, s);
    if (st != HDG_OK) return st;
  }
  TRY(ctx_alloc(c, (void**)&c->e2e, (size_t)c->nel * 4 * sizeof(int32_t)));
  TRY(ctx_alloc(c, (void**)&c->edge_elem, (size_t)c->n_edges * 2 * sizeof(int32_t)));
  TRY(ctx_alloc(c, (void**)&c->edge_face, (size_t)c->n_edges * 2 * sizeof(int32_t)));
  TRY(launch_maps(c, s));
  const int n = c->ref.n, m = c->ref.m;
  TRY(ctx_alloc(c, (void**)&c->Ainv, (size_t)c->nel * n * n * sizeof(double)));
  TRY(ctx_alloc(c, (void**)&c->Gfac, (size_t)c->nel * n * m * sizeof(double)));
  TRY(ctx_alloc(c, (void**)&c->elem_scratch, (size_t)c->nel * m * sizeof(double)));
  if (c->opt.reduced || c->opt.tau_kappa) TRY(ctx_alloc(c, &c->red_z, (size_t)c->nel * m * sizeof(double)));
  // p-levels
  c->plev.resize(k + 1);
  const int spr = (c->mesh.nx + kSeg - 1) / kSeg;
  const bool mixed = c->opt.mixed != 0;
  for (int p = 0; p <= k; ++p) {
    PLevel& L = c->plev[p];
    L.p = p; L.n1 = p + 1; L.m = 4 * (p + 1); L.R = 4 * L.n1 * L.m;
    L.nseg = spr * c->mesh.ny;
    L.rec_entries = (size_t)L.nseg * L.R * kSeg;
    TRY(cudaMallocAsync((void**)&L.Sdense, (size_t)c->nel * L.m * L.m * sizeof(double), s));
    TRY(ctx_alloc(c, (void**)&L.S64, L.rec_entries * sizeof(double)));
    // reduced blocks: for the reduced apply, and with tau_K = kappa_K also for
    // the adjoint gradient (-psi_K^T S_K lambda_K per element)
    if (c->opt.reduced || c->opt.tau_kappa) {
      const size_t ep = ((size_t)c->nel + 31) / 32 * 32;                     // warp chunks
      const size_t Q = (size_t)reduced_entries(L.n1);
      TRY(ctx_alloc(c, (void**)&L.R64, Q * ep * sizeof(double)));
      if (mixed && c->opt.reduced) {
        TRY(ctx_alloc(c, (void**)&L.R32, (Q + 3) / 4 * 4 * ep * sizeof(float)));
        TRY(ctx_alloc(c, (void**)&L.R2, Q * ep * sizeof(float2)));
      }
    }
    if (mixed) {
      TRY(ctx_alloc(c, (void**)&L.S32, L.rec_entries * sizeof(float)));
      TRY(ctx_alloc(c, (void**)&L.S16, L.rec_entries * sizeof(__nv_bfloat16)));
      TRY(ctx_alloc(c, (void**)&L.S2, L.rec_entries * sizeof(float2)));
    }
    if (p >= 1) {
      TRY(ctx_alloc(c, (void**)&L.M64, L.rec_entries * sizeof(double)));
      if (mixed) {
        TRY(ctx_alloc(c, (void**)&L.M32, L.rec_entries * sizeof(float)));
        TRY(ctx_alloc(c, (void**)&L.M16, L.rec_entries * sizeof(__nv_bfloat16)));
        TRY(ctx_alloc(c, (void**)&L.M2, L.rec_entries * sizeof(float2)));
      }
      std::vector<double> Pp;
      p_prolongation_1d(p - 1, Pp);
      TRY(ctx_alloc(c, (void**)&L.Pp, Pp.size() * sizeof(double)));
      TRY(cudaMemcpyAsync(L.Pp, Pp.data(), Pp.size() * sizeof(double), cudaMemcpyHostToDevice, s));
      // float copy for the float V-cycles (a double -> float conversion per use
      // would run on the FP64 pipe)
      const std::vector<float> Pp32(Pp.begin(), Pp.end());
      TRY(ctx_alloc(c, (void**)&L.Pp32, Pp.size() * sizeof(float)));
      TRY(cudaMemcpyAsync(L.Pp32, Pp32.data(), Pp.size() * sizeof(float), cudaMemcpyHostToDevice, s));
      // and the rest P - float(P) for the double-float prolongation into the
      // finest level of a float cycle
      std::vector<float> Pplo(Pp.size());
      for (size_t q = 0; q < Pp.size(); ++q) Pplo[q] = (float)(Pp[q] - (double)Pp32[q]);
      TRY(ctx_alloc(c, (void**)&L.Pplo, Pp.size() * sizeof(float)));
      TRY(cudaMemcpyAsync(L.Pplo, Pplo.data(), Pp.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    }
  }
  TRY(launch_local_setup(c, s));
  {
    // a uniform coefficient makes every element block equal: keep that block for
    // the tensor-core batched apply
    std::vector<double> hk(c->nel);
    TRY(cudaMemcpyAsync(hk.data(), kappa, (size_t)c->nel * sizeof(double), cudaMemcpyDeviceToHost, s));
    TRY(cudaStreamSynchronize(s));
    bool uni = true;
    for (int e = 1; e < c->nel && uni; ++e) uni = (hk[e] == hk[0]);
    c->uniform_kappa = uni;
    // one shared block for every element: S for a uniform kappa, S_ref with a
    // per-element kappa scale when tau_K = kappa_K
    if (uni || c->opt.tau_kappa) TRY(prepare_shared_blocks(c, hk[0], s));
    if (uni && !c->opt.tau_kappa) TRY(prepare_ozaki_blocks(c, s));
  }
  for (int p = k; p >= 1; --p) TRY(launch_galerkin_coarsen(c, p, s));
  for (int p = k; p >= 0; --p) {
    TRY(launch_build_records(c, p, s));
    if (c->opt.reduced || c->opt.tau_kappa) TRY(launch_reduced_blocks(c, p, s));
    if (p >= 1) TRY(launch_asm_blocks(c, p, s));
    if (p >= 1 && c->opt.smoother == 1) TRY(launch_fsai_setup(c, p, s));
  }
  // CG / reduction scratch
  TRY(ctx_alloc(c, (void**)&c->red, 3 * 304 * sizeof(double)));
  TRY(ctx_alloc(c, (void**)&c->scal, 64 * sizeof(double)));
  TRY(cudaMemsetAsync(c->scal, 0, 64 * sizeof(double), s));
  TRY(cudaMallocHost((void**)&c->h_scal, 64 * sizeof(double)));
  const size_t nd = (size_t)c->ndof;
  for (double** p : {&c->cg_r, &c->cg_z, &c->cg_p, &c->cg_q, &c->cg_zold})
    TRY(ctx_alloc(c, (void**)p, nd * sizeof(double)));
  if (c->opt.use_graphs) {   // the device-resident CG loop's iterate, history and control words
    TRY(ctx_alloc(c, (void**)&c->cg_x, nd * sizeof(double)));
    TRY(ctx_alloc(c, (void**)&c->cg_hist, 256 * sizeof(double)));
    TRY(ctx_alloc(c, (void**)&c->cg_ctl, 4 * sizeof(int)));
    TRY(cudaMallocHost((void**)&c->h_cg, 264 * sizeof(double)));
  }
  if (c->opt.autotune) TRY(autotune_applies(c, s));
  TRY(build_hierarchy(c, s));
  TRY(noalloc_prepare_device(c->dev));
  if (c->opt.wait_probe > 0) {
    // armed only now, so the set-up's own applies (autotuning) are not probed
    const int probe = c->opt.wait_probe;
    TRY(cudaMemcpyAsync(c->err_flag + 1, &probe, sizeof(int), cudaMemcpyHostToDevice, s));
  }
  for (int p = 0; p <= k; ++p) {
    TRY(cudaFreeAsync(c->plev[p].Sdense, s));
    c->plev[p].Sdense = nullptr;
  }
  TRY(cudaStreamSynchronize(s));
  return read_err_flag(c, s);
}

int hdg_setup(const hdg_mesh* mesh, int k, const double* kappa, const hdg_options* opt, void* stream,
              void** out_ctx) {
  if (!mesh || !kappa || !out_ctx) return HDG_ERR_INVALID_ARG;
  *out_ctx = nullptr;
  if (k < 0 || k > kMaxDegree) return HDG_ERR_INVALID_ARG;
  if (mesh->nx < 2 || mesh->ny < 2 || mesh->nx > (1 << 15) || mesh->ny > (1 << 15)) return HDG_ERR_INVALID_ARG;
  if (!(mesh->x1 > mesh->x0) || !(mesh->y1 > mesh->y0)) return HDG_ERR_INVALID_ARG;
  hdg_options o;
  hdg_default_options(&o);
  if (opt) o = *opt;
  if (o.nu1 < 1 || o.nu2 < 1 || o.nu1 > 16 || o.nu2 > 16 || o.coarse_n < 2 || !(o.tau > 0.0) ||
      o.cheb_degree < 1 || o.cheb_degree > 8 || o.reduced < 0 || o.reduced > 2 ||
      o.tau_kappa < 0 || o.tau_kappa > 1 || o.wait_probe < 0 || o.wait_probe > 64 || o.smoother < 0 ||
      o.smoother > 1 || o.fmg_start < 0 || o.fmg_start > 16 ||
      o.tensor_apply < 0 || o.tensor_apply > 1 || o.coarse_fuse < 0 || o.coarse_fuse > 1 || o.top_accum < 0 || o.top_accum > 1)
    return HDG_ERR_INVALID_ARG;
  const long nel = (long)mesh->nx * mesh->ny;
  const long ne = (long)(mesh->nx + 1) * mesh->ny + (long)mesh->nx * (mesh->ny + 1);
  if (ne * (k + 1) > 0x7fffffffL) return HDG_ERR_INVALID_ARG;
  Context* c = new (std::nothrow) Context();
  if (!c) return HDG_ERR_OOM;
  c->mesh = *mesh; c->opt = o; c->k = k;
  c->nel = (int)nel; c->n_edges = (int)ne; c->ndof = (int)(ne * (k + 1));
  c->hx = (mesh->x1 - mesh->x0) / mesh->nx;
  c->hy = (mesh->y1 - mesh->y0) / mesh->ny;
  cudaStream_t s = (cudaStream_t)stream;
  const auto t0 = std::chrono::steady_clock::now();
  int st;
  try {
    st = setup_impl(c, kappa, s);
  } catch (...) {
    st = HDG_ERR_INVALID_ARG;
  }
  if (st != HDG_OK) {
    cudaStreamSynchronize(s);
    hdg_destroy(c);
    return st;
  }
  c->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out_ctx = c;
  return HDG_OK;
}

int hdg_get_info(void* ctx, hdg_info* info) {
  Context* c = (Context*)ctx;
  if (!c || !info) return HDG_ERR_INVALID_ARG;
  info->nel = c->nel; info->n_edges = c->n_edges; info->ndof = c->ndof; info->k = c->k;
  info->n_plevels = c->k + 1; info->n_hlevels = (int)c->hlev.size(); info->coarse_dim = c->coarse_dim;
  info->device_bytes = c->bytes; info->setup_ms = c->setup_ms; info->vcycle_kernels = c->vcycle_kernels;
  {
    const bool one_tile = c->mesh.nx <= 32 && c->mesh.ny <= reduced_tile_rows();
    info->apply_kernels = c->opt.reduced == 1 ? 2 : (c->opt.reduced == 2 && !one_tile) ? 2 : 1;
  }
  return HDG_OK;
}

int hdg_get_maps(void* ctx, int32_t* elem_to_edge, int32_t* edge_to_elem, int32_t* edge_local_face, void* stream) {
  Context* c = (Context*)ctx;
  if (!c) return HDG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (elem_to_edge)
    TRY(cudaMemcpyAsync(elem_to_edge, c->e2e, (size_t)c->nel * 4 * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  if (edge_to_elem)
    TRY(cudaMemcpyAsync(edge_to_elem, c->edge_elem, (size_t)c->n_edges * 2 * sizeof(int32_t),
                        cudaMemcpyDeviceToDevice, s));
  if (edge_local_face)
    TRY(cudaMemcpyAsync(edge_local_face, c->edge_face, (size_t)c->n_edges * 2 * sizeof(int32_t),
                        cudaMemcpyDeviceToDevice, s));
  TRY(cudaStreamSynchronize(s));
  return HDG_OK;
}

static bool prec_ok(Context* c, int prec) {
  if (prec == HDG_PREC_FP64) return true;
  if (prec == HDG_PREC_FP32 || prec == HDG_PREC_BF16 || prec == HDG_PREC_F32X2) return c->opt.mixed != 0;
  return false;
}

int hdg_condense_rhs(void* ctx, const double* f_q, double* b, int nrhs, void* stream) {
  Context* c = (Context*)ctx;
  if (!c || !f_q || !b || nrhs < 1) return HDG_ERR_INVALID_ARG;
  TRY(launch_condense(c, f_q, b, nrhs, (cudaStream_t)stream));
  return HDG_OK;
}

int hdg_apply_trace(void* ctx, const void* x, void* y, int nrhs, int prec, void* stream) {
  Context* c = (Context*)ctx;
  if (!c || !x || !y || nrhs < 1 || x == y) return HDG_ERR_INVALID_ARG;
  if (prec < 0 || prec > 3) return HDG_ERR_INVALID_ARG;
  if (!prec_ok(c, prec)) return HDG_ERR_UNSUPPORTED;
  // many right-hand sides on reduced blocks: the scratch of the batched work
  // (allocated on the first call with this nrhs)
  if (nrhs > 1 && c->opt.reduced == 1) {
    const cudaError_t e = use_batched_work(c, nrhs, prec);
    if (e == cudaErrorMemoryAllocation) { cudaGetLastError(); return HDG_ERR_OOM; }
    TRY(e);
  }
  TRY(launch_apply(c, c->k, 0, prec, x, nullptr, y, 1.0, 0.0, nrhs, (cudaStream_t)stream));
  return HDG_OK;
}

int hdg_gmg_vcycle(void* ctx, const void* r, void* z, int nrhs, int prec, void* stream) {
  Context* c = (Context*)ctx;
  if (!c || !r || !z || nrhs < 1) return HDG_ERR_INVALID_ARG;
  if (prec < 0 || prec > 3) return HDG_ERR_INVALID_ARG;
  if (!prec_ok(c, prec)) return HDG_ERR_UNSUPPORTED;
  // nrhs > 1: all columns through one batched cycle (work vectors allocated on first use)
  const cudaError_t e = vcycle(c, prec, r, z, nrhs, (cudaStream_t)stream);
  if (e == cudaErrorMemoryAllocation) { cudaGetLastError(); return HDG_ERR_OOM; }
  TRY(e);
  return HDG_OK;
}

int hdg_setup_batch(int n, const hdg_mesh* meshes, const int* k, const double* const* kappa,
                    const hdg_options* opt, void* stream, void** out) {
  if (n < 1 || n > 16 || !meshes || !k || !kappa || !out) return HDG_ERR_INVALID_ARG;
  for (int q = 0; q < n; ++q) out[q] = nullptr;
  for (int q = 0; q < n; ++q) {
    const int st = hdg_setup(&meshes[q], k[q], kappa[q], opt, stream, &out[q]);
    if (st != HDG_OK) {
      for (int r = 0; r < q; ++r) {
        hdg_destroy(out[r]);
        out[r] = nullptr;
      }
      return st;
    }
  }
  return HDG_OK;
}

int hdg_apply_multi(int n, void* const* ctxs, const void* const* x, void* const* y, int prec, void* stream) {
  if (n < 1 || !ctxs) return HDG_ERR_INVALID_ARG;
  return apply_multi(reinterpret_cast<Context* const*>(ctxs), n, x, y, prec, (cudaStream_t)stream);
}

int hdg_apply_shared_batched(void* ctx, const void* X, float* Y, int nrhs, void* stream) {
  Context* c = (Context*)ctx;
  if (!c || !X || !Y || nrhs < 64 || nrhs % 64 != 0) return HDG_ERR_INVALID_ARG;
  if (((uintptr_t)X % 16) != 0 || ((uintptr_t)Y % 16) != 0) return HDG_ERR_INVALID_ARG;
  if (!c->shared_B) return HDG_ERR_UNSUPPORTED;
  TRY(launch_batched_apply(c, X, Y, nrhs, (cudaStream_t)stream));
  return HDG_OK;
}

int hdg_apply_shared_fp64(void* ctx, const double* X, double* Y, int nrhs, void* stream) {
  Context* c = (Context*)ctx;
  if (!c || !X || !Y || X == Y || nrhs < 64 || nrhs % 64 != 0) return HDG_ERR_INVALID_ARG;
  if (((uintptr_t)X % 16) != 0 || ((uintptr_t)Y % 16) != 0) return HDG_ERR_INVALID_ARG;
  if (!c->oz_B) return HDG_ERR_UNSUPPORTED;
  const cudaError_t e = launch_ozaki_apply(c, X, Y, nrhs, (cudaStream_t)stream);
  if (e == cudaErrorMemoryAllocation) { cudaGetLastError(); return HDG_ERR_OOM; }
  TRY(e);
  return HDG_OK;
}

int hdg_solve(void* ctx, const double* b, double* lambda, int nrhs, double rtol, int maxit, int inner,
              hdg_solve_info* info, void* stream) {
  Context* c = (Context*)ctx;
  if (!c || !b || !lambda || nrhs < 1 || !(rtol > 0.0) || maxit < 1 || b == lambda) return HDG_ERR_INVALID_ARG;
  if (inner < 0 || inner > 3) return HDG_ERR_INVALID_ARG;
  if (!prec_ok(c, inner)) return HDG_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  const auto t0 = std::chrono::steady_clock::now();
  int st = nrhs == 1 ? pcg_solve(c, b, lambda, rtol, maxit, inner, info, s)
                     : pcg_solve_batched(c, b, lambda, nrhs, rtol, maxit, inner, info, s);
  const int fl = read_err_flag(c, s);
  // a wait that gave up leaves part of an apply unwritten, which can also stop
  // CG from converging: report the cause
  if (fl != HDG_OK && (st == HDG_OK || st == HDG_ERR_NOT_CONVERGED || st == HDG_ERR_BREAKDOWN)) st = fl;
  if (info) info->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return st;
}

int hdg_recover_local(void* ctx, const double* lambda, const double* f_q, double* u, double* q, void* stream) {
  Context* c = (Context*)ctx;
  if (!c || !lambda || !f_q) return HDG_ERR_INVALID_ARG;
  if (!u && !q) return HDG_OK;
  TRY(launch_recover(c, lambda, f_q, u, q, (cudaStream_t)stream));
  return HDG_OK;
}

int hdg_fmg(void* ctx, const double* b, double* lambda, int cycles, void* stream) {
  Context* c = (Context*)ctx;
  if (!c || !b || !lambda || b == lambda || cycles < 1 || cycles > 16) return HDG_ERR_INVALID_ARG;
  const cudaError_t e = fmg_solve(c, b, lambda, cycles, (cudaStream_t)stream);
  if (e == cudaErrorMemoryAllocation) { cudaGetLastError(); return HDG_ERR_OOM; }
  TRY(e);
  return HDG_OK;
}

int hdg_postprocess(void* ctx, const double* u, const double* q, double* ustar, double* qstar, void* stream) {
  Context* c = (Context*)ctx;
  if (!c || !u || !q) return HDG_ERR_INVALID_ARG;
  if (!ustar && !qstar) return HDG_OK;
  TRY(launch_postprocess(c, u, q, ustar, qstar, (cudaStream_t)stream));
  return HDG_OK;
}

__global__ void residual_interior_kernel(int nx, int ny, int n1, const double* __restrict__ a,
                                         const double* __restrict__ b, double* __restrict__ out) {
  const int nv = (nx + 1) * ny, ne = nv + nx * (ny + 1);
  const size_t total = (size_t)ne * n1;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int ed = (int)(t / n1);
    bool interior;
    if (ed < nv) { const int i = ed % (nx + 1); interior = i > 0 && i < nx; }
    else { const int j = (ed - nv) / nx; interior = j > 0 && j < ny; }
    out[t] = interior ? a[t] - b[t] : 0.0;
  }
}
__global__ void half_kernel(const double* in, double* out) { out[0] = 0.5 * in[0]; }

int hdg_adjoint_grad(void* ctx, const double* f_q, const double* lambda, const double* lambda_obs, double rtol,
                     int maxit, double* dJ_dlogk, double* dJ_df, double* J, double* psi, void* stream) {
  Context* c = (Context*)ctx;
  if (!c || !f_q || !lambda || !lambda_obs || !(rtol > 0.0) || maxit < 1) return HDG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = (size_t)c->ndof;
  double *res, *ps;
  TRY(cudaMallocAsync((void**)&res, n * sizeof(double), s));
  TRY(cudaMallocAsync((void**)&ps, n * sizeof(double), s));
  int blocks = (int)((n + 255) / 256);
  if (blocks > 2048) blocks = 2048;
  residual_interior_kernel<<<blocks, 256, 0, s>>>(c->mesh.nx, c->mesh.ny, c->k + 1, lambda, lambda_obs, res);
  TRY(cudaGetLastError());
  if (J) {
    TRY(vec_dot(c, res, res, (int)n, c->scal + 32, s));
    half_kernel<<<1, 1, 0, s>>>(c->scal + 32, J);
    TRY(cudaGetLastError());
  }
  hdg_solve_info info;
  int st = pcg_solve(c, res, ps, rtol, maxit, HDG_PREC_FP64, &info, s);
  if (st == HDG_OK) {
    cudaError_t e = launch_adjoint(c, f_q, lambda, ps, dJ_dlogk, dJ_df, s);
    if (e != cudaSuccess) st = map_cuda(e);
  }
  if (st == HDG_OK && psi) {
    cudaError_t e = cudaMemcpyAsync(psi, ps, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) st = map_cuda(e);
  }
  cudaFreeAsync(res, s);
  cudaFreeAsync(ps, s);
  const int fl = read_err_flag(c, s);
  if (st == HDG_OK && fl != HDG_OK) st = fl;
  return st;
}

void hdg_destroy(void* ctx) {
  Context* c = (Context*)ctx;
  if (!c) return;
  cudaDeviceSynchronize();
  release_works(c);
  for (auto& L : c->plev)
    if (L.Sdense) cudaFree(L.Sdense);
  for (void* p : c->allocs) cudaFree(p);
  if (c->oz_XS) cudaFree(c->oz_XS);
  if (c->oz_ecol) cudaFree(c->oz_ecol);
  if (c->h_scal) cudaFreeHost(c->h_scal);
  delete c;
}

}  // extern "C"
