/*
 * hdg.h -- C ABI of the GB300 library for the statically condensed HDG trace
 * operator of -div(kappa grad u) = f (u = 0 on the boundary) on a uniform
 * Cartesian quad mesh, and the nested p/h geometric multigrid built on it.
 *
 * Method: Fabien, Knepley, Mills, Riviere, "Manycore parallel computing for a
 * hybridizable discontinuous Galerkin nested multigrid method" (arXiv
 * 1705.09907). Section, equation and algorithm numbers below refer to it.
 *
 * Conventions shared by every call
 *  - Mesh: nx x ny rectangles on [x0,x1] x [y0,y1]; element e = i + nx*j.
 *    Edges: vertical ones first, id = i + (nx+1)*j (i in [0,nx], j in [0,ny));
 *    then horizontal ones, id = (nx+1)*ny + i + nx*j (i in [0,nx), j in [0,ny]).
 *    Local faces of an element: 0 = W, 1 = E, 2 = S, 3 = N.
 *  - Trace vectors ("x", "y", "b", "lambda"): [n_edges][k+1] values at the k+1
 *    Gauss-Legendre nodes of each edge, ordered by increasing coordinate;
 *    dof = edge*(k+1) + a. With nrhs > 1 the layout is [n_edges*(k+1)][nrhs]
 *    (right-hand side fastest). Entries on boundary edges are outputs of 0 and
 *    are ignored on input (the trace is P_h g_D = 0 there).
 *  - Source samples f_q: [nel][k+2][k+2], f at the (k+2)^2 Gauss-Legendre points
 *    of each element, index [e][jy][ix] (x fastest).
 *  - Volume output u: [nel][(k+1)^2], q: [nel][2][(k+1)^2] -- values at the
 *    tensor Gauss-Lobatto nodes, index i + (k+1)*j (i along x); k = 0: the
 *    element constant.
 *  - All vector arguments are DEVICE pointers owned by the caller, unless a
 *    name says host. The context owns everything it allocates.
 *  - `stream` is a cudaStream_t passed as void* (0 = legacy default stream).
 *    Calls are asynchronous on that stream unless they return host-visible
 *    results (hdg_setup, hdg_solve, hdg_adjoint_grad, hdg_get_*), which
 *    synchronise it.
 *  - Every call returns an hdg_status. On an error nothing is written to the
 *    outputs that later calls depend on; the context stays usable unless the
 *    status is HDG_ERR_CUDA (a sticky CUDA error).
 *  - A context holds work vectors, scratch and captured V-cycle graphs that its
 *    calls reuse: calls on one context must not run concurrently (issue them
 *    from one thread, or on one stream in order). Different contexts are
 *    independent.
 *  - The FP32 / BF16 / F32X2 precisions below describe the blocks a call
 *    reads. With `hdg_options.reduced` (default) the condensed blocks are read
 *    in their symmetry-reduced form: FP64 and F32X2 calls use the FP64 reduced
 *    blocks, FP32 and BF16 calls the FP32 reduced blocks; the Schwarz blocks of
 *    the V-cycle are always read in the precision named.
 */
#ifndef HDG_H
#define HDG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HDG_OK = 0,
  HDG_ERR_INVALID_ARG = 1,   /* bad size, degree, pointer or option          */
  HDG_ERR_CUDA = 2,          /* a CUDA runtime call or kernel launch failed  */
  HDG_ERR_OOM = 3,           /* device allocation failed                     */
  HDG_ERR_NOT_CONVERGED = 4, /* iteration limit reached before the tolerance */
  HDG_ERR_BREAKDOWN = 5,     /* CG breakdown: p^T A p <= 0 or not finite     */
  HDG_ERR_TIMEOUT = 6,       /* a bounded device wait gave up                */
  HDG_ERR_UNSUPPORTED = 7    /* valid request this build does not provide    */
} hdg_status;

/* Storage / arithmetic precision of an operator apply or V-cycle.
 *  FP64:  blocks and vectors in double, double accumulation.
 *  FP32:  blocks and vectors in float, float accumulation.
 *  BF16:  blocks in bfloat16, vectors in float, float accumulation.
 *  F32X2: blocks as pairs of floats (hi + lo, about 48 significant bits),
 *         vectors in double, products and sums in compensated ("double-float")
 *         FP32 arithmetic: FP64-class results from the FP32 pipe, whose rate on
 *         this GPU is about 60x the FP64 rate.
 * FP32 and BF16 apply the condensed blocks to x minus its mean on each element
 * (exact in exact arithmetic because every S_K has zero row sums). */
typedef enum { HDG_PREC_FP64 = 0, HDG_PREC_FP32 = 1, HDG_PREC_BF16 = 2, HDG_PREC_F32X2 = 3 } hdg_prec;

typedef struct {
  int nx, ny;                 /* elements per direction, >= 1                */
  double x0, y0, x1, y1;      /* domain corners, x1 > x0, y1 > y0            */
} hdg_mesh;

typedef struct {
  int nu1, nu2;               /* pre/post smoothing steps (2, 2), Algs. 1-2  */
  int coarse_n;               /* coarsen the Q1 meshes while both sizes are even
                                 and halving keeps them >= coarse_n (2)       */
  double tau;                 /* HDG stabilisation on every facet (1.0)      */
  int cheb_degree;            /* Chebyshev degree per h-level smoothing step (2) */
  int mixed;                  /* also build FP32, BF16 and F32X2 copies of the
                                 level blocks (1)                             */
  int use_graphs;             /* capture V-cycles in CUDA graphs, and run the
                                 iterations of a one-right-hand-side hdg_solve
                                 as one graph launch (a conditional WHILE node
                                 whose body ends in the stopping test: no host
                                 round trip per iteration, the same iterates
                                 as the host loop); 0: host loop and direct
                                 launches (1)                                 */
  int autotune;               /* 1: time the apply kernels (the ring kernel's
                                 launch shapes and the one-CTA-per-segment
                                 kernel) per level and precision at set-up and
                                 keep the fastest (default); 0: the ring kernel
                                 with its default shape; 2 / 3 / 4: the
                                 segment kernel with 8 / 4 / 2 warps wherever it
                                 fits. The
                                 choice changes only the
                                 order of the floating-point sums            */
  int reduced;                /* 1: one-vector applies of the condensed blocks
                                 use each S_K reduced by the element's two
                                 reflection symmetries (four symmetric blocks,
                                 61 numbers instead of 400 at k = 4), in two
                                 launches: element products, then faces
                                 (default); 2: the same arithmetic and results
                                 with one CTA per 32 x 8 element tile plus a
                                 small launch for the faces on tile edges;
                                 0: the dense owner records (kernel chosen by
                                 `autotune`). With 1 or 2, double vectors in
                                 F32X2 use the reduced blocks as float pairs
                                 in double-float arithmetic, and one-vector
                                 FP32 Schwarz applies use the Schwarz blocks
                                 packed as symmetric upper triangles (element
                                 pass + face pass)                          */
  int tau_kappa;              /* 1: tau_K = kappa_K on the faces of element K
                                 (tau piecewise constant per element, Sec. 3;
                                 `tau` is unused): every local equation then
                                 scales with kappa_K, S_K = kappa_K S_ref and
                                 the condensed right-hand side does not depend
                                 on kappa; 0: tau = `tau` everywhere (0)     */
  int smoother;               /* p-level smoother of the V-cycle: 0 = weighted
                                 additive Schwarz on element patches
                                 (Sec. 6.4.2, default); 1 = factorized sparse
                                 approximate inverse (Sec. 6.4.1), x += G^T G
                                 (f - A x), G lower triangular on the pattern
                                 of the level operator, unit diagonal of
                                 G A G^T                                      */
  int tensor_apply;           /* 1: hdg_solve with nrhs a multiple of 64 (at
                                 most 2048) applies the outer operator of the
                                 batched CG on the tensor cores in FP64 by
                                 exact slice splitting (hdg_apply_shared_fp64)
                                 when every element shares one block (uniform
                                 kappa, tau not tied to kappa, k <= 7); its
                                 slices of the CG direction are scratch of the
                                 context (16 bytes per entry); 0: the CUDA-core
                                 column kernels (1)                           */
  int fmg_start;              /* hdg_solve with one right-hand side starts CG
                                 from one full multigrid cycle (Sec. 7) with
                                 this many V-cycles per level instead of from
                                 zero; 0 = zero start (0), at most 16         */
  size_t max_device_bytes;    /* cap on the device memory the context keeps
                                 (set-up data and work vectors; 0 = no cap):
                                 an allocation that would pass it fails with
                                 HDG_ERR_OOM as if the device were full (0)   */
  int wait_probe;             /* test of the bounded-wait path (0 = off): the
                                 first `wait_probe` launches after set-up of
                                 the one-CTA-per-segment apply kernel (see
                                 `autotune`) make their first CTA wait, with
                                 the usual ~1 s bound, on a barrier nothing
                                 completes; it gives up, raises the context's
                                 error flag, drains its own block copy and
                                 exits, so the call that reads the flag
                                 (hdg_solve, hdg_adjoint_grad) returns
                                 HDG_ERR_TIMEOUT; later calls run normally.
                                 0 <= wait_probe <= 64                        */
  int coarse_fuse;            /* 1: the coarse Q1 levels run as one single-CTA
                                 kernel per V-cycle: from the first level
                                 whose stencils and vectors, with every
                                 coarser level's, fit in one CTA's shared
                                 memory, smoothing, residuals, transfers and
                                 the coarsest solve (through the inverse of
                                 its Cholesky factorisation, when it has at
                                 most 1024 unknowns) are phases of one launch
                                 (default); 0: one launch per step on every
                                 level                                        */
  int top_accum;              /* 1: FP32 / BF16 V-cycles keep the finest
                                 level's correction as a double-float pair
                                 (two floats, ~48 bits) and prolongate into it
                                 in double-float arithmetic; every operator of
                                 the cycle stays in float, BF16 cycles use the
                                 FP32 blocks on the finest level and the BF16
                                 blocks below: the iteration counts of FP64
                                 cycles (default); 0: the correction in float,
                                 BF16 blocks on every p-level                */
} hdg_options;

typedef struct {
  int nel, n_edges, ndof;     /* ndof = n_edges * (k+1)                      */
  int k, n_plevels, n_hlevels;/* p-levels k..0 and Q1 h-levels (finest first) */
  int coarse_dim;             /* unknowns of the coarsest (direct) solve     */
  size_t device_bytes;        /* device memory held by the context           */
  double setup_ms;            /* wall time of hdg_setup                      */
  int vcycle_kernels;         /* kernel launches in one V-cycle (0 until the
                                 first V-cycle has been captured or run)     */
  int apply_kernels;          /* kernel launches of one hdg_apply_trace of
                                 one vector (2 with `reduced` = 1, and with 2
                                 on meshes of more than one tile; else 1)    */
} hdg_info;

typedef struct {
  int iterations;             /* CG iterations taken                         */
  double relres;              /* final |r|_2 / |b|_2, r the residual CG
                                 updates (FP64 vectors); a recomputed b - A x
                                 differs by rounding, ~eps |A||x| per row,
                                 which grows like h^-2 relative to |b|        */
  double relres_history[256]; /* per iteration, [0] = 1                       */
  double solve_ms;            /* wall time of the call                       */
} hdg_solve_info;

/* Fill `opt` with the defaults listed above. */
void hdg_default_options(hdg_options* opt);

/* Human-readable text for a status code (static storage). */
const char* hdg_error_string(int status);

/*
 * Build the solver for degree k (0 <= k <= 7) and per-element coefficient
 * kappa (device, [nel] doubles, each > 0 and finite; K = kappa*I, piecewise
 * constant as in Sec. 2). Performs procedure (i) of Sec. 3 -- the local
 * solvers of Eq. shur0 and the condensed blocks S_K of Eq. shur1 on every
 * element -- then the multigrid hierarchy of Sec. 6: Galerkin p-levels k-1..0,
 * Schwarz blocks, the conforming Q1 h-levels with Galerkin coarsening, the
 * Chebyshev bounds, and the FP64 Cholesky factor of the coarsest operator.
 * `opt` may be NULL (defaults). On success *out owns all device data; release
 * it with hdg_destroy. Errors: INVALID_ARG (sizes, k, kappa <= 0 or NaN, bad
 * options), OOM, CUDA.
 */
int hdg_setup(const hdg_mesh* mesh, int k, const double* kappa, const hdg_options* opt,
              void* stream, void** out_ctx);

/* Sizes and setup statistics (host struct). */
int hdg_get_info(void* ctx, hdg_info* info);

/*
 * Index maps (device outputs, int32): elem_to_edge [nel][4] (faces W,E,S,N),
 * edge_to_elem [n_edges][2] (low-side, high-side element; -1 off the domain),
 * edge_local_face [n_edges][2] (face of the edge in those elements; -1).
 * These are the maps Map0..Map3 of Alg. 3. Any output may be NULL.
 */
int hdg_get_maps(void* ctx, int32_t* elem_to_edge, int32_t* edge_to_elem,
                 int32_t* edge_local_face, void* stream);

/*
 * Condensed right-hand side (Sec. 3 step (ii); the volume-to-surface
 * projection of Sec. 8.3): b = sum_K A_K^T b_K, b_K(mu) = (f, u_mu)_K.
 * f_q: device [nrhs][nel][k+2][k+2] doubles; b: device [ndof][nrhs] doubles
 * (nrhs = 1: [ndof]). Boundary entries of b are written as 0.
 */
int hdg_condense_rhs(void* ctx, const double* f_q, double* b, int nrhs, void* stream);

/*
 * Assembly-free apply of the condensed trace operator (Alg. 3):
 * y_e = sum over the two elements K of edge e of S_K[e rows, :] x_K on every
 * interior edge, y = 0 on boundary edges. Each face is written once, by one
 * thread, with no atomics. x, y: device [ndof][nrhs] in the type `prec`
 * selects (double for FP64 and F32X2, float for FP32 and BF16); x and y must
 * not overlap. Kernels: with `reduced` (default) the symmetry-reduced blocks
 * (one vector: element pass + face pass; nrhs > 1 with double vectors: the
 * column form of the same, bitwise equal per column, whose scratch belongs to
 * the batched work of that nrhs, allocated by the first call with it); else,
 * and for float columns, the dense owner records (nrhs > 1: each CTA stages one
 * segment's blocks in shared memory once and applies them to all columns).
 * Errors: INVALID_ARG (nrhs < 1, null pointers), UNSUPPORTED (FP32/BF16/F32X2
 * when the context was built with mixed = 0), OOM (batched work).
 */
int hdg_apply_trace(void* ctx, const void* x, void* y, int nrhs, int prec, void* stream);

/*
 * Set up n independent problems of uneven size and degree in one call (the
 * instances of hdg_apply_multi): out[q] receives the context of mesh meshes[q],
 * degree k[q] and coefficient kappa[q] (device, [nx*ny] doubles each), with the
 * same options for all (opt may be NULL). Same validation and errors as
 * hdg_setup for each instance; on any error every context created by this call
 * is destroyed, all out[q] are NULL, and the first failing instance's status is
 * returned. 1 <= n <= 16.
 */
int hdg_setup_batch(int n, const hdg_mesh* meshes, const int* k, const double* const* kappa,
                    const hdg_options* opt, void* stream, void** out);

/*
 * The trace apply of Alg. 3 for n independent meshes (1 <= n <= 16 contexts,
 * uneven sizes, degrees 0..5) as one batch: the work of all meshes forms a
 * single list (each CTA serves one mesh, on its degree), so small meshes do not
 * leave SMs idle behind large ones. When every context has `reduced` = 1 the
 * batch is the element pass and the face pass of the reduced apply, one launch
 * each for all meshes (each result bitwise equal to the mesh's own apply);
 * otherwise one launch over all record segments of the dense owner records.
 * y[q] = A_q x[q] for each q, same layouts and boundary rules
 * as hdg_apply_trace (nrhs = 1). prec: HDG_PREC_FP64 (double vectors) or
 * HDG_PREC_FP32 (float vectors). All contexts must belong to the current device.
 * Errors: INVALID_ARG (count, pointers, degree, device), UNSUPPORTED (FP32 when a
 * context has no FP32 blocks, other precisions).
 */
int hdg_apply_multi(int n, void* const* ctxs, const void* const* x, void* const* y, int prec, void* stream);

/*
 * Batched apply with one shared element block: Y = A X for nrhs right-hand
 * sides on the 5th-generation tensor cores, for a uniform coefficient (every
 * S_K equal) or for tau_K = kappa_K (every S_K = kappa_K S_ref, Sec. 3 with tau
 * piecewise constant; each element's part scaled by its kappa when the
 * accumulator is read). Each owned face computes
 * y_e = s_K S[F rows] x_K + s_nb S[F' rows] x_nb (Alg. 3 with a shared block) as one
 * MMA row block: two faces x 64 right-hand sides (M = 128) by the 2*4(k+1)
 * gathered dofs (K) by 16 outputs (N: the own element's k+1 rows, then the
 * neighbour's), FP32 accumulation in tensor memory. X: device BF16
 * [ndof][nrhs] (right-hand side fastest), Y: device FP32 [ndof][nrhs]; nrhs a
 * multiple of 64; both 16-byte aligned; boundary entries of X are ignored and Y
 * is 0 there. X is read through TMA tensor maps made for each call. Errors:
 * INVALID_ARG (nrhs, alignment, null), UNSUPPORTED (neither a uniform kappa
 * nor tau_kappa).
 */
int hdg_apply_shared_batched(void* ctx, const void* X, float* Y, int nrhs, void* stream);

/*
 * FP64 batched apply for a uniform coefficient on the BF16 tensor cores, by
 * exact integer splitting (the Ozaki scheme): Y = A X with X, Y device FP64
 * [ndof][nrhs] (right-hand side fastest), nrhs a multiple of 64, 16-byte
 * aligned, X and Y distinct. Each column of X is scaled by a power of two and
 * cut into 8 BF16 slices of 7 bits (56 bits in all), the shared element block
 * likewise at set-up; the products of slices are exact in the tensor cores'
 * FP32 accumulation and the groups of equal weight are recombined as 128-bit
 * integers and rounded once to FP64, so the result agrees with an FP64
 * evaluation to about the FP64 rounding of |S||x| (terms below 2^-56 of the
 * column's and the block's scale are dropped; entries below 2^-1022 count as
 * zero). Same face formula, boundary rules and layouts as
 * hdg_apply_shared_batched. The slices of X (8 x 2 bytes per entry) are
 * scratch owned by the context, grown on demand. Errors: INVALID_ARG,
 * UNSUPPORTED (kappa not uniform, tau_kappa, or k > 7), OOM.
 */
int hdg_apply_shared_fp64(void* ctx, const double* X, double* Y, int nrhs, void* stream);

/*
 * One nested V-cycle z = V r (Algs. 2 then 1, zero initial guess): p-levels
 * k..1 with nu1/nu2 weighted additive Schwarz steps (Sec. 6.4.2), restriction
 * R = P^T and prolongation P per edge (Eqs. eq_mg_pro, eq_mg_res), the p = 0
 * level and the Q1 levels with Chebyshev steps, P_J / P_J^T between p = 0 and
 * Q1 (Eq. eq_h_mg_pro), bilinear transfers, and an FP64 Cholesky solve on the
 * coarsest mesh. r, z: device [ndof][nrhs] (double for FP64 and F32X2, float
 * for FP32 and BF16; the Q1 levels run in the vector type, the coarsest solve
 * in FP64).
 * With nrhs > 1 every level works on all columns at once; the work vectors for
 * that nrhs are allocated on the first such call (and replaced when nrhs
 * changes), and the cycle is captured as its own CUDA graph. Errors: OOM when
 * those vectors do not fit.
 * The operator is symmetric positive definite, so CG may use it.
 */
int hdg_gmg_vcycle(void* ctx, const void* r, void* z, int nrhs, int prec, void* stream);

/*
 * Solve A lambda = b (Sec. 3 step (iii)) with conjugate gradients
 * preconditioned by one V-cycle per iteration, until the updated residual
 * satisfies |r|_2 <= rtol |b|_2.
 * b, lambda: device [ndof][nrhs] doubles (right-hand side fastest). With
 * nrhs > 1 the columns iterate together: one batched operator apply and one
 * batched V-cycle per iteration, step lengths per column, and a column stops
 * updating once its own residual meets rtol; info then reports the iteration
 * at which the last column converged and the largest residual. The CG vectors, the
 * update and the residual are FP64 vectors; `inner` selects the V-cycle
 * precision. With inner = FP64 every apply is plain FP64. With inner = FP32,
 * BF16 or F32X2 the outer operator apply uses F32X2 blocks (FP64 vectors,
 * ~48-bit products) and CG uses the flexible Polak-Ribiere beta, since a
 * low-precision V-cycle is not exactly symmetric. info (host, may be NULL) receives the
 * iteration count and residual history. Errors: NOT_CONVERGED (lambda holds
 * the last iterate), BREAKDOWN, TIMEOUT (a bounded device wait gave up during
 * the solve; reported in preference to NOT_CONVERGED or BREAKDOWN, which it
 * may have caused), CUDA.
 */
int hdg_solve(void* ctx, const double* b, double* lambda, int nrhs, double rtol, int maxit,
              int inner, hdg_solve_info* info, void* stream);

/*
 * n independent problems of uneven size solved together (1 <= n <= 64
 * contexts, e.g. from hdg_setup_batch, all on the current device, each at most
 * once): hdg_solve of context q on (b[q], lambda[q]) with the common rtol,
 * maxit and inner precision. With use_graphs on in every context (and no
 * fmg_start) all instances form one CUDA graph launched once: per instance a
 * chain of its set-up kernels, a conditional WHILE node iterating its CG and
 * the copy of its solution, the chains independent, so the instances share
 * the GPU at the same time (small meshes fill the SMs that large ones leave
 * idle) with no host round trip until all have finished; otherwise each runs
 * on a stream and host thread of its own. Every instance runs the kernels of
 * its own hdg_solve, so each lambda[q] is bitwise what hdg_solve gives for it
 * alone. The call
 * orders itself after the work already issued on `stream`, makes `stream` wait
 * for every instance, and returns when all have finished. b[q], lambda[q]:
 * device [ndof_q] doubles. infos (host [n], may be NULL) and statuses (host
 * [n], may be NULL) receive each instance's report and status; the return
 * value is HDG_OK if every instance converged, else the first failing
 * instance's status. Errors: INVALID_ARG (count, pointers, a context twice or
 * on another device), UNSUPPORTED (a mixed precision without mixed blocks),
 * and those of hdg_solve.
 */
int hdg_solve_multi(int n, void* const* ctxs, const double* const* b, double* const* lambda, double rtol,
                    int maxit, int inner, hdg_solve_info* infos, int* statuses, void* stream);

/*
 * Surface-to-volume reconstruction (Sec. 3 step (iv), Eq. shur0, Sec. 8.3):
 * from the trace lambda [ndof] and sources f_q [nel][k+2][k+2] compute
 * u [nel][(k+1)^2] and q [nel][2][(k+1)^2] (device doubles; either may be NULL).
 */
int hdg_recover_local(void* ctx, const double* lambda, const double* f_q, double* u, double* q,
                      void* stream);

/*
 * One full multigrid cycle (Sec. 7): b (device [ndof] doubles) restricted to
 * every level (R = P^T), a direct solve on the coarsest mesh, then level by
 * level upwards the coarser solution interpolated (P) as the start and
 * `cycles` FP64 V-cycles of that level's own hierarchy (Alg. 1 on the p = 0
 * and Q1 levels, Alg. 2 on the p-levels) applied to its residual; lambda
 * (device [ndof]) receives the finest solution. Asynchronous on `stream`. Its
 * per-level vectors are allocated on the first call. 1 <= cycles <= 16.
 * Errors: INVALID_ARG, OOM.
 */
int hdg_fmg(void* ctx, const double* b, double* lambda, int cycles, void* stream);

/*
 * Element-local postprocessing (Sec. 3 step (v); the local filter of the LDG-H
 * analysis the paper cites, Sec. 5 and Table 1): on each element K, u* in
 * Q_{k+1}(K) solves the Neumann problem (kappa grad u*, grad w)_K =
 * -(q_h, grad w)_K for all w in Q_{k+1}(K) with the element mean of u_h, and
 * q* = -kappa grad u*. u*, q* converge at rates k+2 and k+1 (Table 1).
 * u [nel][(k+1)^2], q [nel][2][(k+1)^2]: device inputs in the layout of
 * hdg_recover_local. ustar [nel][(k+2)^2], qstar [nel][2][(k+2)^2]: device
 * outputs, values at the (k+2)^2 tensor Gauss-Lobatto nodes of each element
 * (index i + (k+2)*j, i along x); either may be NULL. Errors: INVALID_ARG.
 */
int hdg_postprocess(void* ctx, const double* u, const double* q, double* ustar, double* qstar, void* stream);

/*
 * Adjoint gradient of J = 1/2 |lambda - lambda_obs|_2^2 (interior dofs) where
 * lambda solves A(kappa) lambda = b(kappa, f). Solves A psi = lambda - lambda_obs
 * with the same multigrid-preconditioned CG (A is symmetric) to rtol, then an
 * element-local kernel gives
 *   dJ/dlog(kappa_K) = -(kappa^-1 q_K(lambda, f), q_K(psi, 0))_K
 *   dJ/df at the sample points = w_q |J_K| u_K(psi, 0)(x_q)
 * with (q, u) from the local solver of Eq. shur0.
 * f_q, lambda, lambda_obs: device inputs; dJ_dlogk [nel], dJ_df [nel][k+2][k+2],
 * J (one double), psi [ndof]: device outputs, each may be NULL.
 */
int hdg_adjoint_grad(void* ctx, const double* f_q, const double* lambda, const double* lambda_obs,
                     double rtol, int maxit, double* dJ_dlogk, double* dJ_df, double* J,
                     double* psi, void* stream);

/*
 * hdg_condense_rhs without any device allocation, for callers that cannot
 * allocate device memory when they need the right-hand side (code running
 * where an allocation would synchronise the device or is not permitted).
 * The paper has no counterpart; this is a library-interface addition.
 * Same arguments, layout and result as hdg_condense_rhs. Its per-element
 * scratch is a fixed array of 2^19 doubles (4 MiB) inside the library, held
 * by every GPU that loads the library until the process exits; contexts
 * with nel * 4(k+1) > 2^19 are rejected with HDG_ERR_INVALID_ARG. hdg_setup
 * looks up that array's device address on the context's device (this loads
 * the part of the library that holds it), so calls made afterwards on that
 * device find it ready and do no host-side set-up; the address does not
 * survive a cudaDeviceReset (which also ends every context). The call must be
 * made with the context's device current (else HDG_ERR_INVALID_ARG). All
 * calls share the array: calls that overlap on the GPU (different streams, no
 * ordering between them) race on it and must not be issued. The array needs
 * no clearing: every call overwrites the entries it reads. Allocates nothing
 * (no cudaMalloc, no cudaFree, no allocating library routine).
 */
int hdg_condense_rhs_noalloc(void* ctx, const double* f_q, double* b, int nrhs, void* stream);

/* Release everything the context owns. NULL is ignored. */
void hdg_destroy(void* ctx);

#ifdef __cplusplus
}
#endif
#endif /* HDG_H */
