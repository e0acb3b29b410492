// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstddef>
#include <vector>
#include <string>

#include "../../include/hdg.h"

namespace hdg {

constexpr int kMaxDegree = 7;
constexpr int kSeg = 16;          // elements per record segment (x direction)

// ---------------------------------------------------------------------------
// Host reference tables for one degree p on an hx x hy rectangle.
// Volume basis: Lagrange at the (p+1)^2 tensor Gauss-Lobatto nodes (p >= 1) or
// the constant (p = 0); trace basis: Lagrange at the p+1 Gauss-Legendre nodes.
// All matrices are row-major doubles.
struct RefTables {
  int p = 0, n1 = 1, n = 1, m = 4, nf = 4;  // nf = (p+2)^2 source samples
  double hx = 1, hy = 1;
  // Local solver pieces (Eq. shur0 after eliminating q):
  //   A_u = kappa*P + tau*Mb   [n x n]
  //   W   = kappa*Z + tau*Eb   [n x m]
  //   S   = kappa*Y + tau*diag(Ml) - W^T A_u^-1 W   [m x m]
  std::vector<double> P, Mb, Z, Eb, Y, Ml;
  std::vector<double> M;                    // volume mass [n x n]
  // Recovery of q: q_c = kappa * (MiBt_c U - MiC_c lambda), c = x, y
  std::vector<double> MiBt, MiC;            // [2][n x n], [2][n x m]
  // Source load F = Vf^T (wJf .* f_q)
  std::vector<double> Vf, wJf;              // [nf x n], [nf]
};

void build_ref_tables(int p, double hx, double hy, RefTables& t);
// Postprocessing tables (hdg_basis.cpp): Hq [2][ns][n], mu [n], Dn [2][ns][ns],
// ns = (p+2)^2
void build_post_tables(int p, double hx, double hy, std::vector<double>& Hq, std::vector<double>& mu,
                       std::vector<double>& Dn);
// Per-edge embedding degree p -> p+1: Pp[(p+2) x (p+1)], Pp[a'][a] = mu_a(x_a')
void p_prolongation_1d(int p, std::vector<double>& Pp);
// 1-D Gauss-Legendre and Gauss-Lobatto rules (ascending nodes)
void gauss_legendre(int q, std::vector<double>& x, std::vector<double>& w);
void gauss_lobatto(int q, std::vector<double>& x, std::vector<double>& w);

// ---------------------------------------------------------------------------
// Device data of one p-level. Blocks are kept in the "owner record" layout:
// segment s = row j, elements i0..i0+15 of that row; each element holds the row
// blocks needed to compute its W and S faces:
//   slot 0: S_K[W rows, :]        slot 1: S_{K-1}[E rows, :]   (west neighbour)
//   slot 2: S_K[S rows, :]        slot 3: S_{K-nx}[N rows, :]  (south neighbour)
// entry r = (slot*(p+1) + a)*m + c, stored at [(seg*R + r)*16 + lane].
struct PLevel {
  int p = 0, n1 = 1, m = 4, R = 16;
  int nseg = 0;
  size_t rec_entries = 0;                   // nseg * R * 16
  double* S64 = nullptr; float* S32 = nullptr; __nv_bfloat16* S16 = nullptr;
  double* M64 = nullptr; float* M32 = nullptr; __nv_bfloat16* M16 = nullptr;
  float* Mp32 = nullptr;                    // Schwarz blocks as packed upper triangles (float cycles)
  float2* S2 = nullptr; float2* M2 = nullptr;   // double-float (hi, lo) copies
  // condensed blocks reduced by the element's reflection symmetry: packed
  // upper triangles of the four character blocks, [Q][nel] (apply_reduced.cu)
  double* R64 = nullptr; float* R32 = nullptr;
  float2* R2 = nullptr;                     // reduced blocks as (hi, lo) float pairs (F32X2 applies)
  double* Sdense = nullptr;                 // [nel][m][m] FP64 element blocks
  double* Pp = nullptr;                     // prolongation from p-1 [(p+1) x p] (device)
  float* Pp32 = nullptr;                    // the same in float (float V-cycles)
  float* Pplo = nullptr;                    // Pp - Pp32 in float (double-float prolongation)
  // V-cycle work vectors, [ndof] each, per precision (d = double, f = float)
  double *r64 = nullptr, *x64 = nullptr, *t64 = nullptr, *d64 = nullptr;
  float *r32 = nullptr, *x32 = nullptr, *t32 = nullptr, *d32 = nullptr;
  // FSAI smoother (hdg_options.smoother = 1, p >= 1): factor G by row edge and
  // slot (hdg_fsai.cu), FP64 and FP32; w: scratch of G t for one vector
  double* G64 = nullptr; float* G32 = nullptr;
  size_t fsai_entries = 0;
  double* w64 = nullptr; float* w32 = nullptr;
  // p = 0 only: inverse diagonal of the assembled operator (Chebyshev/Jacobi)
  double* dinv64 = nullptr; float* dinv32 = nullptr;
  double lmax = 0.0;
  int tune[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};   // apply launch shape per (prec, S/M)
};

// One Q1 level (interior vertices (nx-1) x (ny-1)); 9-point stencils stored as
// [9][nv] with offsets (dx, dy) in {-1,0,1}^2, index (dy+1)*3 + (dx+1).
struct HLevel {
  int nx = 0, ny = 0, nv = 0;
  double* st64 = nullptr; float* st32 = nullptr;
  float* rsum32 = nullptr;                  // row sums (difference-form float apply)
  double* dinv64 = nullptr; float* dinv32 = nullptr;
  double lmax = 0.0;
  double *r64 = nullptr, *x64 = nullptr, *t64 = nullptr, *d64 = nullptr, *e64 = nullptr;
  float *r32 = nullptr, *x32 = nullptr, *t32 = nullptr, *d32 = nullptr, *e32 = nullptr;   // e: second direction
};

// Work vectors of one V-cycle in one vector type (double for FP64 / F32X2
// cycles, float for FP32 / BF16 cycles) for nb right-hand sides stored
// right-hand-side fastest ([n][nb]). The single-vector work points into the
// levels' own buffers; a batched work owns its buffers (and the batched CG
// vectors of hdg_solve with nrhs > 1).
struct VWork {
  int nb = 1;
  bool dbl = true;
  std::vector<void*> pr, px, pt;            // p-levels 0..k: residual, correction, scratch
  std::vector<void*> pw;                    // p-levels 0..k: FSAI scratch (null without FSAI)
  void* p0d = nullptr;                      // p = 0 Chebyshev direction
  std::vector<void*> hr, hx, ht, hd, hd2;   // Q1 levels, finest first (hd2: second Chebyshev direction)
  double* coarse_w = nullptr;               // [nb][coarse_dim] FP64 scratch
  cudaGraphExec_t graph[4] = {nullptr, nullptr, nullptr, nullptr};   // per precision
  cudaStream_t gstream[4] = {nullptr, nullptr, nullptr, nullptr};
  // batched CG (double works only): vectors [ndof][nb], per-column scalars, partials
  double *cg_r = nullptr, *cg_z = nullptr, *cg_p = nullptr, *cg_q = nullptr, *cg_zold = nullptr;
  double* cg_sc = nullptr;                  // [kCgScalars][nb]
  double* cg_part = nullptr;                // [3][reduction blocks][nb]
  double* h_sc = nullptr;                   // pinned host mirror [2][nb]
  std::vector<void*> own;                   // device buffers owned by this work
  size_t own_bytes = 0;                     // their total size
  size_t cap = ~size_t(0);                  // most it may allocate (memory cap)
  void* red_z = nullptr;                    // batched reduced-apply scratch [4(k+1)][nel][nb]
  // float cycles: low part of the finest level's correction (its high part is
  // px[k]) and a float scratch of that level ([ndof][nb] each; null: the
  // correction is accumulated in float)
  float* top_lo = nullptr;
  float* top_u = nullptr;
};

// Per-level vectors of the full multigrid cycle (double, one right-hand side):
// right-hand side, solution, residual and correction on every p-level and Q1 level
struct FmgWork {
  bool ready = false;
  std::vector<double*> bp, xp, rp, zp;      // p-levels 0..k
  std::vector<double*> bh, xh, rh, zh;      // Q1 levels, finest first
};

struct Context {
  hdg_mesh mesh{};
  hdg_options opt{};
  int k = 0, nel = 0, n_edges = 0, ndof = 0;
  int dev = 0, num_sms = 0;
  int smem_optin = 0;                       // max dynamic shared memory per block (opt-in)
  double hx = 0, hy = 0;
  double* kappa = nullptr;                  // [nel] (copy)
  int32_t* e2e = nullptr;                   // [nel][4]
  int32_t* edge_elem = nullptr;             // [n_edges][2]
  int32_t* edge_face = nullptr;             // [n_edges][2]
  RefTables ref;                            // finest degree
  double* d_ref = nullptr;                  // device copy of the finest tables
  size_t off_P = 0, off_Mb = 0, off_Z = 0, off_Eb = 0, off_Y = 0, off_Ml = 0,
         off_MiBt = 0, off_MiC = 0, off_Vf = 0, off_wJf = 0, off_M = 0;
  size_t off_ZT = 0, off_EbT = 0, off_MiBtT = 0, off_MiCT = 0, off_VfT = 0;   // transposes
  double* elem_scratch = nullptr;           // [nel][m] per-element partial results
  double* d_post = nullptr;                 // postprocessing tables: Hq^T [2][n][ns], mu [n], Dn^T [2][ns][ns]
  int* fsai_rowslots = nullptr;             // FSAI apply tables [n_edges][6] (hdg_fsai.cu)
  int* fsai_colrows = nullptr;
  int post_ns = 0;                          // (k+2)^2
  void* red_z = nullptr;                    // [m][nel] element products of the reduced apply
  // finest-level local operators: A_u^-1 (symmetric, stored full) and G = A_u^-1 W
  double* Ainv = nullptr;                   // [nel][n][n]
  double* Gfac = nullptr;                   // [nel][n][m]
  std::vector<PLevel> plev;                 // index p = 0..k
  std::vector<HLevel> hlev;                 // finest Q1 first
  double* coarse_L = nullptr;               // dense FP64 Cholesky factor [nc][nc]
  double* coarse_AinvT = nullptr;           // its inverse, transposed (fused coarse cycle; nc <= 1024)
  float *top_lo32 = nullptr, *top_u32 = nullptr;   // the single float work's top_lo, top_u
  int coarse_dim = 0;
  double* coarse_rhs = nullptr;             // [nc] FP64 scratch
  // CG / reduction scratch
  double* red = nullptr;                    // partial sums
  double* scal = nullptr;                   // device scalars
  double* h_scal = nullptr;                 // pinned host mirror
  double *cg_r = nullptr, *cg_z = nullptr, *cg_p = nullptr, *cg_q = nullptr, *cg_zold = nullptr;
  float* cg_r32 = nullptr;
  float* cg_z32 = nullptr;
  int* err_flag = nullptr;                  // device error flag (timeouts)
  // device-resident CG loop (one graph per inner precision, built on first use)
  cudaGraphExec_t cg_graph[4] = {nullptr, nullptr, nullptr, nullptr};
  bool cg_graph_failed = false;             // conditional graphs unavailable: host loop
  double* cg_x = nullptr;                   // the loop's iterate
  double* cg_hist = nullptr;                // relative residual per iteration [256]
  int* cg_ctl = nullptr;                    // iterations, status, maxit
  double* h_cg = nullptr;                   // pinned host copy of the loop's results [264]
  size_t bytes = 0;
  double setup_ms = 0.0;
  std::vector<void*> allocs;
  // V-cycle work: single vector (double, float family) and batched (on demand)
  VWork w1[2];                              // [0] double, [1] float
  FmgWork fmg;                              // full multigrid work (first hdg_fmg call)
  VWork* wb[2] = {nullptr, nullptr};
  // the reduced-apply scratch of the batched work whose cycle, solve or apply
  // is being issued (launch_apply with nrhs > 1 uses it; null: dense columns)
  void* cur_zb = nullptr;
  size_t cur_zb_bytes = 0;
  int vcycle_kernels = 0;                   // kernel nodes of the captured V-cycle
  // uniform coefficient: the shared block for the tensor-core batched apply
  bool uniform_kappa = false;
  __nv_bfloat16* shared_B = nullptr;        // [2][16][Kp] BF16
  bool shared_scaled = false;               // shared_B is S_ref (tau_K = kappa_K): scale by kappa_K
  // FP64 shared-block apply by integer splitting (hdg_ozaki.cu): the block's
  // BF16 slices [8][2][16][64] and exponent, the slices of X and the column
  // exponents (scratch of the last nrhs, grown on demand)
  uint16_t* oz_B = nullptr;
  int oz_eS = 0;
  void* oz_XS = nullptr;
  size_t oz_xs_bytes = 0;
  int* oz_ecol = nullptr;
  int oz_ecol_n = 0;
};

// vectors of a V-cycle / apply in this precision are double (else float)
inline bool prec_double(int prec) { return prec == HDG_PREC_FP64 || prec == HDG_PREC_F32X2; }

// allocation helper: records the pointer for hdg_destroy
cudaError_t ctx_alloc(Context* c, void** p, size_t bytes);

// ---------------------------------------------------------------------------
// Kernel entry points (implemented in the .cu files)
cudaError_t launch_local_setup(Context* c, cudaStream_t s);
cudaError_t launch_galerkin_coarsen(Context* c, int p_fine, cudaStream_t s);
cudaError_t launch_build_records(Context* c, int p, cudaStream_t s);
cudaError_t launch_asm_blocks(Context* c, int p, cudaStream_t s);
cudaError_t launch_p0_diag(Context* c, cudaStream_t s);
cudaError_t autotune_applies(Context* c, cudaStream_t s);
// tensor-core batched apply of the shared block (hdg_batched.cu)
cudaError_t prepare_shared_blocks(Context* c, double kappa0, cudaStream_t s);
cudaError_t launch_batched_apply(Context* c, const void* X, float* Y, int nrhs, cudaStream_t s);
// FP64 shared-block apply on the tensor cores by exact splitting (hdg_ozaki.cu)
cudaError_t prepare_ozaki_blocks(Context* c, cudaStream_t s);
cudaError_t launch_ozaki_apply(Context* c, const double* X, double* Y, int nrhs, cudaStream_t s);
// one persistent launch over several contexts (apply_multi.cu); returns hdg_status
int apply_multi(Context* const* ctx, int n, const void* const* x, void* const* y, int prec, cudaStream_t s);

// Reduced-block apply (apply_reduced.cu): entries per element of the packed
// blocks, their set-up from the dense blocks, and y = beta c + alpha S v for one
// vector (two launches).
int reduced_entries(int n1);
int reduced_tile_rows();                  // rows of one tile of the reduced apply
cudaError_t launch_reduced_blocks(Context* c, int p, cudaStream_t s);
cudaError_t launch_reduced_apply(Context* c, int p, int prec, const void* v, const void* cvec, void* y,
                                 double alpha, double beta, cudaStream_t s);
// the same for nb right-hand sides ([ndof][nb]) with the scratch z of
// nel * 4(p+1) * nb vector entries (a batched work's)
cudaError_t launch_reduced_cols(Context* c, int p, int prec, const void* v, const void* cvec, void* y, double alpha,
                                double beta, int nb, void* z, cudaStream_t s);
// dth_K = -psi_K^T S_K lambda_K per element at level k (the adjoint gradient
// with tau_K = kappa_K)
cudaError_t launch_reduced_theta(Context* c, const double* lam, const double* psi, double* dth, cudaStream_t s);

// Trace-operator apply on the record layout of level p:
//   y = beta * cvec + alpha * (B v), B = S (which = 0) or Schwarz M (which = 1)
// vectors in double (prec FP64) or float (FP32/BF16); cvec may be null.
// Schwarz blocks of the float cycles as packed upper triangles (from the dense
// per-element blocks Md at set-up), and their apply y = beta c + alpha M v
cudaError_t launch_sym_pack(Context* c, int p, const double* Md, cudaStream_t s);
cudaError_t launch_sym_schwarz(Context* c, int p, const void* v, const void* cvec, void* y, double alpha,
                               double beta, cudaStream_t s);
cudaError_t launch_apply(Context* c, int p, int which, int prec, const void* v, const void* cvec,
                         void* y, double alpha, double beta, int nrhs, cudaStream_t s);

// Multigrid pieces (hdg_mg.cu)
cudaError_t build_hierarchy(Context* c, cudaStream_t s);
// z = V r for nb right-hand sides ([ndof][nb]; double for FP64 / F32X2, float otherwise)
cudaError_t vcycle(Context* c, int prec, const void* r, void* z, int nb, cudaStream_t s);
int pcg_solve(Context* c, const double* b, double* x, double rtol, int maxit, int inner,
              hdg_solve_info* info, cudaStream_t s);
// one graph for several contexts' one-right-hand-side solves (hdg_solve_multi):
// add one instance's chain, then after the launch fetch and read its results
cudaError_t cg_multi_add(Context* c, int inner, const double* b, double* lambda, double rtol, int maxit, cudaGraph_t G,
                         cudaStream_t cs);
cudaError_t cg_multi_fetch(Context* c, cudaStream_t s);
int cg_multi_result(Context* c, hdg_solve_info* info);
// CG on nb right-hand sides at once (b, x: [ndof][nb]), one V-cycle of all
// columns per iteration, per-column step lengths; a column stops updating once
// its residual meets rtol
int pcg_solve_batched(Context* c, const double* b, double* x, int nb, double rtol, int maxit, int inner,
                      hdg_solve_info* info, cudaStream_t s);
// one full multigrid cycle with `cycles` FP64 V-cycles per level: x = FMG(b)
cudaError_t fmg_solve(Context* c, const double* b, double* x, int cycles, cudaStream_t s);
// releases the V-cycle works' graphs and the batched works' buffers
void release_works(Context* c);
// makes the batched work of nb right-hand sides (vector type of prec) current
// for column applies: allocates it on first use, sets cur_zb
cudaError_t use_batched_work(Context* c, int nb, int prec);

// FSAI smoother (hdg_fsai.cu): factor of level p from plev[p].Sdense, and
// out = add + G^T G in for nb columns (add may be null or alias out)
cudaError_t launch_fsai_setup(Context* c, int p, cudaStream_t s);
cudaError_t launch_fsai_smooth(Context* c, int p, int prec, const void* in, const void* add, void* out, void* wbuf,
                               int nb, cudaStream_t s);

// Vector helpers (hdg_apply.cu)
cudaError_t vec_dot(Context* c, const double* a, const double* b, int n, double* out_dev, cudaStream_t s);
cudaError_t vec_fill(void* p, int prec, size_t n, cudaStream_t s);

// looks up the allocation-free scratch of hdg_condense_rhs_noalloc on device
// dev (current) at set-up (hdg_noalloc.cu)
cudaError_t noalloc_prepare_device(int dev);

// Local element operations (hdg_local.cu)
cudaError_t launch_condense(Context* c, const double* f_q, double* b, int nrhs, cudaStream_t s);
cudaError_t launch_recover(Context* c, const double* lam, const double* f_q, double* u, double* q,
                           cudaStream_t s);
cudaError_t launch_adjoint(Context* c, const double* f_q, const double* lam, const double* psi,
                           double* dJ_dlogk, double* dJ_df, cudaStream_t s);
// u* and q* of the element-local postprocessing (hdg_post.cu)
cudaError_t launch_postprocess(Context* c, const double* u, const double* q, double* ustar, double* qstar,
                               cudaStream_t s);

}  // namespace hdg

#define HDG_CUDA_TRY(expr)                                  \
  do {                                                      \
    cudaError_t _e = (expr);                                \
    if (_e != cudaSuccess) return _e;                       \
  } while (0)
