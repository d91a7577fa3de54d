/*
 * libbem: GB300 (sm_103a) frequency-domain elastodynamic boundary element
 * method with the exponential window (EWM) and frequency-domain windowing.
 *
 * Method: Xiao, Ye, Wen, "Efficiency improvement of the frequency-domain BEM
 * for rapid transient elastodynamic analysis".
 *   Sec. 2.1  problem (Eq. governing-pde), BIE (Eq. bie), kernels (Eqs. Uij,
 *             Tij, Gikj), constant-element collocation T u = U t (Eq. Tu_Ut),
 *             boundary conditions A a = b (Eq. Aa_b)
 *   Sec. 2.2  sampling relations T = 2 pi / dw, dt = T / N, solve k = 0..N/2
 *   Sec. 3    exponential window s_k = eta + i k dw, windows, DFT-MFT and
 *             IDFT-MFT (Eqs. DFT-MFT, IDFT-MFT)
 *   Sec. 4    the sequence A_k a_k = b_k (Eq. Aa_b-sequence), solution
 *             extrapolation (Eqs. a0, lsem, a0-solution)
 *   Sec. 5    block-diagonal preconditioned GMRES, tolerance 1e-5
 *
 * Conventions for every entry point:
 *   - Returns BEM_OK (0) or a negative BEM_ERR_* code; bem_last_error()
 *     gives a one-line message. No entry point aborts or exits the process.
 *   - All pointers without the _dev suffix are HOST pointers owned by the
 *     caller; the library copies what it needs during the call and keeps no
 *     caller pointer after returning. *_dev pointers are DEVICE pointers on
 *     the context's device, borrowed for the duration of the call.
 *   - Complex arrays are interleaved (re, im) float64 pairs.
 *   - Unknown/dof numbering: dof = 3 * element + component, in the caller's
 *     element order.
 *   - One context = one device and one stream; calls on one context must not
 *     overlap. Work is enqueued on the context's stream; every call that
 *     returns host data synchronises that stream.
 *   - The library allocates the device memory it needs (cudaMalloc) and frees
 *     it in bem_destroy.
 */
#ifndef BEM_H_
#define BEM_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BEM_OK 0
#define BEM_ERR_INVALID_ARG (-1)
#define BEM_ERR_NO_MESH (-2)
#define BEM_ERR_OOM (-3)
#define BEM_ERR_CUDA (-4)
#define BEM_ERR_NOT_CONVERGED (-5)
#define BEM_ERR_TIMEOUT (-6) /* reserved: no entry point returns it (no call waits on the device) */
#define BEM_ERR_STATE (-7)

/* element boundary-condition kind (Sec. 2.1: Gamma_sigma / Gamma_u) */
#define BEM_BC_TRACTION 0     /* traction prescribed, displacement unknown */
#define BEM_BC_DISPLACEMENT 1 /* displacement prescribed, traction unknown */

/* frequency-domain windows (Sec. 3.2) */
#define BEM_WIN_NONE 0
#define BEM_WIN_HANNING 1
#define BEM_WIN_BLACKMAN 2

/* operator precision */
#define BEM_PREC_C64_MIXED 0 /* complex64 operator and Krylov basis, FP32 kernel
                                evaluation; FP64 singular/near-singular
                                integrals, Arnoldi dots, Givens, true-residual
                                refinement */
#define BEM_PREC_C128 1      /* complex128 everywhere (the plain form) */

/* initial guess of each frequency system */
#define BEM_GUESS_ZERO 0
#define BEM_GUESS_SEM 1 /* least-squares solution extrapolation (Sec. 4.2) */
#define BEM_GUESS_MLP 2 /* Sec. 4.2 extrapolation over the previous solutions
                           plus one learned proposal column (bem_mlp_*); the
                           paper has no learned guess */

/* storage of the far-field factors (bem_set_far_storage) */
#define BEM_FAR_AUTO 0    /* full when both operator sets' capped factors take at
                             most a quarter of the device memory, else compact */
#define BEM_FAR_FULL 1    /* every block's U, V at its rank cap, ACA writes in place */
#define BEM_FAR_COMPACT 2 /* ACA in a workspace batch by batch, factors packed at
                             their actual ranks; a sweep keeps a second operator
                             set (the next frequency assembled during the solve)
                             only where it fits in a fifth of the free memory */

/* block-diagonal preconditioner of GMRES (Sec. 3.1, Sec. 5: "block diagonal",
 * block size not stated) */
#define BEM_PRECOND_BLOCK3 0 /* the 3 x 3 diagonal block of each element (default) */
#define BEM_PRECOND_LEAF 1   /* the diagonal block of each cluster-tree leaf (up to
                                64 elements: 192 x 192), inverted per frequency; needs
                                leaf_size <= 64 */
#define BEM_PRECOND_AUTO 2   /* a sweep solves its first frequency with k > 0 with
                                both and keeps the one that took fewer GMRES steps */

typedef struct bem_ctx bem_ctx;

typedef struct bem_opts {
  double tol;         /* true relative residual ||b - A a|| / ||b|| (Sec. 5: 1e-5) */
  int32_t restart;    /* GMRES restart length m (paper: unstated; default 50) */
  int32_t max_iters;  /* Arnoldi steps per frequency before NOT_CONVERGED */
  double aca_tol;     /* ACA stopping tolerance of far-field blocks */
  int32_t leaf_size;  /* cluster-tree leaf size in elements (default 64) */
  double eta_adm;     /* admissibility: min(diam) <= eta_adm * dist */
  int32_t precision;  /* BEM_PREC_* */
  int32_t guess;      /* BEM_GUESS_* */
  int32_t sem_k;      /* K previous solutions for the extrapolation (Sec. 4.2: 3-4) */
  int32_t dense;      /* 1: every block dense (no ACA); for small meshes and tests */
  int32_t precond;    /* BEM_PRECOND_* (Sec. 5: block diagonal; block size unstated) */
} bem_opts;

typedef struct bem_freq_stats {
  int32_t k;              /* frequency index */
  int32_t iters;          /* Arnoldi steps used */
  int32_t cycles;         /* restart cycles (each starts from an FP64 true residual) */
  int32_t converged;      /* 1 if rel_residual <= tol */
  double s_re, s_im;      /* s_k = eta + i k dw */
  double rel_residual;    /* final true relative residual, FP64 accumulation */
  double guess_residual;  /* ||b - A a0|| / ||b|| of the initial guess */
  double assemble_ms;     /* operator + right-hand side */
  double guess_ms;
  double solve_ms;
  int64_t near_bytes;     /* bytes of dense near-field blocks */
  int64_t far_bytes;      /* bytes of low-rank factors actually used */
  int32_t max_rank;
  int32_t aca_failures;   /* far blocks that hit the rank cap */
  double sem_residual;    /* least-squares residual ||b - A a0|| / ||b|| of the
                             extrapolation over the previous solutions alone
                             (products in the operator's precision); with
                             BEM_GUESS_MLP, compare with guess_residual to see
                             what the learned column added; 1 without a guess */
  int32_t precond;        /* BEM_PRECOND_BLOCK3 or BEM_PRECOND_LEAF: the one the
                             accepted solve used */
  int32_t trial_iters;    /* BEM_PRECOND_AUTO: Arnoldi steps of the comparison
                             solve with the other preconditioner (included in
                             iters); 0 otherwise */
} bem_freq_stats;

/* Fill *opts with the defaults: tol 1e-5, restart 50, max_iters 5000,
 * aca_tol 1e-5, leaf 64, eta_adm 1.0, mixed precision, SEM guess, K 4. */
void bem_default_opts(bem_opts* opts);

/* Create a context on CUDA device `device`, enqueuing on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream). */
int bem_create(bem_ctx** out, int device, void* cuda_stream);
void bem_destroy(bem_ctx* ctx);
const char* bem_last_error(const bem_ctx* ctx);

/* Surface mesh of the solid (Sec. 2.1, constant triangles, Eq. Tu_Ut).
 * xyz: nv x 3 vertex coordinates; tri: ne x 3 vertex indices, with
 * (v1 - v0) x (v2 - v0) pointing OUT of the solid (into cavities);
 * bc_type: ne values BEM_BC_*. Replaces any previous mesh; builds element
 * geometry, the cluster tree and the frequency-independent static (Kelvin)
 * parts of the singular and near-singular integrals.
 * Errors: INVALID_ARG (sizes, index out of range, degenerate triangle). */
int bem_mesh(bem_ctx* ctx, const double* xyz, int64_t nv, const int32_t* tri, int64_t ne,
             const int8_t* bc_type, const bem_opts* opts);
/* Same with device-resident inputs. */
int bem_mesh_dev(bem_ctx* ctx, const double* xyz_dev, int64_t nv, const int32_t* tri_dev,
                 int64_t ne, const int8_t* bc_type_dev, const bem_opts* opts);

/* Isotropic material (Sec. 2.1): E > 0, -1 < nu < 0.5, rho > 0. */
int bem_set_material(bem_ctx* ctx, double E, double nu, double rho);

/* Exponential-window damping eta >= 0 (Sec. 3.1; Eq. ewm-k gives
 * eta = kappa ln 10 / T) and frequency window BEM_WIN_* (Sec. 3.2). */
int bem_set_window(bem_ctx* ctx, double eta, int window);

/* Solve the whole sequence A_k a_k = b_k, k = 0..n_omega/2 (Eq.
 * Aa_b-sequence) at s_k = eta + i k 2 pi / T. The prescribed data is
 * separable: value(element, component, t) = bc_pattern[3e+c] * P(t), with
 * load_hist[n] = P(n T / n_omega), n = 0..n_omega-1, transformed by Eq.
 * DFT-MFT. bc_pattern: ne x 3 (traction on Gamma_sigma elements,
 * displacement on Gamma_u elements). stats (optional): n_omega/2 + 1
 * entries. n_omega must be even and >= 2.
 * The assemblies of the next frequencies overlap the solve of frequency k
 * (up to two ahead with full far-field storage, in operator sets of their
 * own); GMRES is driven by the device (its rotations, convergence test and
 * restarts run in kernels); the call returns once the whole sweep is done.
 * Errors: NO_MESH, STATE (material not set), INVALID_ARG, NOT_CONVERGED
 * (every frequency is still solved as far as max_iters allows and stored). */
int bem_solve_sweep(bem_ctx* ctx, double T, int32_t n_omega, const double* load_hist,
                    const double* bc_pattern, const bem_opts* opts, bem_freq_stats* stats);
int bem_solve_sweep_dev(bem_ctx* ctx, double T, int32_t n_omega, const double* load_hist_dev,
                        const double* bc_pattern_dev, const bem_opts* opts,
                        bem_freq_stats* stats);

/* Solution a_k of frequency k (N = 3 ne complex values; displacement at
 * Gamma_sigma elements, traction at Gamma_u elements). */
int bem_get_frequency_solution(bem_ctx* ctx, int32_t k, double* out);

/* Time response R(n dt), n = 0..n_omega-1, at the given dofs by Eq.
 * IDFT-MFT with the context's window, the spectrum extended by conjugate
 * symmetry (Sec. 2.2 step 3; the k = 0 and k = n_omega/2 samples enter by
 * their real parts). out: n_omega x ndof row-major float64. */
int bem_time_response(bem_ctx* ctx, const int64_t* dofs, int64_t ndof, double* out);
/* Same, device output (n_omega x ndof float64) and device dof list. */
int bem_time_response_dev(bem_ctx* ctx, const int64_t* dofs_dev, int64_t ndof, double* out_dev);

/* ---- interior field ----------------------------------------------------
 * Displacement and strain at points inside the solid from the solved
 * boundary data, by the representation formula (Somigliana's identity: the
 * interior form of Eq. bie, free term c = I; Sec. 5.2 reports strain at an
 * interior point of its plate example):
 *   u_i(x) = sum_e [ int_e U_ij(x, y) dy t_j(e) - int_e T_ij(x, y) dy u_j(e) ],
 * u, t constant per element: the solved values a_k and the prescribed
 * pattern * P_k, placed by each element's boundary condition. Each
 * (point, element) pair uses the rule of its distance band, as the operator
 * entries do (the nearest band: the full kernel on the 1,024-point
 * subdivided rule). Kernel evaluation in the operator's precision (FP32 for
 * the complex64 operator, FP64 for complex128), geometry relative to the
 * point in FP64, sums in FP64.
 * points: npts x 3 float64 (caller coordinates). Points must lie inside the
 * solid at a distance from the boundary (at least a fraction of the local
 * element size); on the boundary the formula does not hold and the values
 * are not finite. Strain: eps = (grad u + grad u^T) / 2 by central
 * differences with step h (the six points x +- h e_a must also be inside).
 * Requires a solved sweep (STATE otherwise); k indexes its frequencies. */
#define BEM_FIELD_DISPLACEMENT 0 /* 3 components: u_x, u_y, u_z */
#define BEM_FIELD_STRAIN 1       /* 6 components: xx, yy, zz, xy, yz, xz */
/* out: npts x 3 complex (interleaved float64). */
int bem_interior_field(bem_ctx* ctx, int32_t k, const double* points, int64_t npts, double* out);
/* out: npts x 6 complex (interleaved float64). */
int bem_interior_strain(bem_ctx* ctx, int32_t k, const double* points, int64_t npts, double h, double* out);
/* Time histories by Eq. IDFT-MFT over every solved frequency, with the
 * context's window: out n_omega x (npts x ncomp) row-major float64, ncomp = 3
 * (BEM_FIELD_DISPLACEMENT) or 6 (BEM_FIELD_STRAIN, step h). */
int bem_interior_time_response(bem_ctx* ctx, const double* points, int64_t npts, int32_t quantity, double h,
                               double* out);

/* ---- step-level entry points (each is one step of the sweep) ---------- */

/* Eq. DFT-MFT: out[k], k = 0..n_omega/2 (complex) of P(n dt). */
int bem_load_dft(bem_ctx* ctx, double T, int32_t n_omega, double eta, const double* load_hist,
                 double* out);

/* Eq. IDFT-MFT on an arbitrary spectrum: Rk is (n_omega/2+1) x ndof complex,
 * out is n_omega x ndof float64. */
int bem_idft(bem_ctx* ctx, double T, int32_t n_omega, double eta, int window, const double* Rk,
             int64_t ndof, double* out);

/* Build the operator A(s) (near-field blocks, ACA far-field blocks, block
 * preconditioner) at the complex frequency s. */
int bem_assemble(bem_ctx* ctx, double s_re, double s_im, const bem_opts* opts);

/* Rows of the assembled operator: out is nrows x N complex (dense rows,
 * far-field entries reconstructed from the low-rank factors). */
int bem_operator_rows(bem_ctx* ctx, const int64_t* rows, int64_t nrows, double* out);

/* y = M^-1 x with the assembled operator's block-diagonal preconditioner
 * (Sec. 3.1, Sec. 5): BEM_PRECOND_BLOCK3, the inverses of the 3 x 3 diagonal
 * blocks (FP64), or BEM_PRECOND_LEAF, the inverses of the leaves' diagonal
 * blocks (complex64 operator: FP32 Gauss-Jordan; complex128: FP64), which
 * need an assembly with precond = BEM_PRECOND_LEAF (STATE otherwise).
 * x, y: N complex (caller order). */
int bem_apply_preconditioner(bem_ctx* ctx, int32_t precond, const double* x, double* y);
/* y = A x with the assembled operator (FP64 accumulation). x, y: N complex. */
int bem_apply(bem_ctx* ctx, const double* x, double* y);

/* Right-hand side b = p * B(s) pattern of Eq. Aa_b at the assembled s,
 * where B has the U columns of Gamma_sigma elements and -T (free term
 * included) columns of Gamma_u elements. pattern: ne x 3 real. */
int bem_rhs(bem_ctx* ctx, double p_re, double p_im, const double* pattern, double* b);

/* Solve A(s) x = b at the assembled s by block-Jacobi GMRES; x0 may be NULL
 * (zero guess). */
int bem_solve_assembled(bem_ctx* ctx, const double* b, const double* x0, double* x,
                        const bem_opts* opts, bem_freq_stats* stats);

/* Solution extrapolation (Sec. 4.2) at the assembled s: a0 = X s with
 * s = argmin ||A X s - b||; X is K x N complex (rows = previous solutions). */
int bem_sem_guess(bem_ctx* ctx, int32_t K, const double* X, const double* b, double* a0);

/* y = A x with the operator assembled by bem_assemble (complex64, mixed
 * precision), for callers that cannot allocate device memory during a call:
 * a framework whose caching allocator has reserved the device's memory up
 * front, or a solver loop with hard latency bounds that cannot take the
 * implicit synchronisation of cudaMalloc/cudaFree. The paper has no
 * counterpart; this is a service entry point of the library.
 *   x_dev, y_dev: DEVICE arrays of N complex64 values (interleaved float
 *   re, im), caller's dof order, allocated by the caller; y must not alias x.
 * The call allocates nothing: its scratch (two permuted vectors, the V^T x
 * values of the low-rank blocks and the partial row sums) is one file-scope
 * device array of 32 MiB that every GPU loading the library holds until the
 * process exits. Operators whose scratch would exceed it are rejected with
 * BEM_ERR_INVALID_ARG (the message gives the sizes). The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) and
 * should come before any stream capture. All calls share the one array and
 * the last call's contents remain in it (nothing needs to start at zero):
 * calls that overlap on the GPU, from any context or stream, race. The work
 * is enqueued on the context's stream; the call does not synchronise it.
 * Errors: STATE (not assembled, or complex128 operator), INVALID_ARG. */
int bem_apply_noalloc(bem_ctx* ctx, const float* x_dev, float* y_dev);

/* Cross-frequency reuse of the ACA pivots (default on). The paper assembles
 * every frequency from scratch; with reuse, each assembly after the first on
 * a mesh starts every admissible block from the pivot rows and columns ACA
 * chose at the previous assembly: it evaluates them at the new s, forms the
 * cross approximation through them (an LU of the r x r pivot block without
 * pivoting), keeps the leading pivots that are still within a factor 10 of
 * their residual row's largest entry, applies ACA's stopping test
 * |u_l| |v_l| <= aca_tol ||S_l||_F to the reused steps, and continues with
 * ACA steps where it is not met. ACA records two spare pivots past its
 * stopping point (their factor columns are stored but not used), so that a
 * block whose rank grows by one or two between frequencies is settled by
 * the reuse alone. */
int bem_set_aca_reuse(bem_ctx* ctx, int on);
/* Admissible blocks of the current mesh after the last assembly: *count =
 * number of blocks; for the first min(nmax, count) blocks info[4b..4b+3] =
 * rows (elements), columns (elements), rank, and the rank the reused pivots
 * settled on their own (equal to the rank when no ACA step was needed; -1
 * when the last assembly did not reuse pivots). nmax = 0 queries the count.
 * Errors: STATE (not assembled). */
int bem_far_block_info(bem_ctx* ctx, int64_t nmax, int32_t* info, int64_t* count);

/* Far-field factor storage of the meshes set after this call (mode
 * BEM_FAR_AUTO, _FULL or _COMPACT). The admissible blocks' factors at their
 * rank caps (3 min(rows, cols) elements, at most 512 columns) need
 * 3 (rows + cols) x cap complex entries per block: at 231k elements that is far
 * above the device memory, though ACA stops at a fraction of the cap. Compact
 * storage runs ACA over consecutive runs of blocks (batches) whose capped
 * factors fit a workspace of `workspace_bytes` (0: 8 GiB for complex64,
 * 16 GiB for complex128, raised to the largest block when smaller) and
 * packs each block's first `rank` columns of U and V into pools that grow
 * by a quarter over the need when an assembly overflows them (the assembly
 * is then redone from the same pivot state, so the result does not depend
 * on the pools' history). Both storages give bit-identical operators.
 * Errors: INVALID_ARG. */
int bem_set_far_storage(bem_ctx* ctx, int32_t mode, int64_t workspace_bytes);

/* The block partition bem_mesh builds, on the host alone (no device, no
 * context): centroid (ne x 3) and element size h (ne, the longest edge) in
 * caller order; leaf_size, eta_adm and dense as in bem_opts. The cluster tree
 * halves each cluster at the median along the longest extent of its
 * centroids until at most leaf_size remain; a cluster pair is admissible
 * (far, low rank) when min(diam) <= eta_adm dist (bounding boxes of the
 * centroids) and dist^2 > 2.2 h_max^2 (no element pair of it in the
 * near-singular band); the other leaf pairs are near. perm (may be NULL):
 * ne values, tree position -> caller element. near_blocks / far_blocks: the
 * first nmax blocks as (row begin, rows, column begin, columns) in tree
 * positions, 4 int32 each; *n_near, *n_far the counts (nmax = 0 queries
 * them). Errors: INVALID_ARG. */
int bem_block_tree(const double* centroid, const double* h, int64_t ne, int32_t leaf_size, double eta_adm,
                   int32_t dense, int32_t* perm, int64_t nmax, int32_t* near_blocks, int32_t* far_blocks,
                   int64_t* n_near, int64_t* n_far);

typedef struct bem_far_storage {
  int32_t compact;          /* storage of the current mesh: 1 compact, 0 full */
  int32_t batches;          /* ACA batches per assembly */
  int64_t workspace_bytes;  /* compact: workspace allocated for the last assembly */
  int64_t factor_bytes;     /* U and V storage allocated for the set in use */
  int64_t used_bytes;       /* U and V bytes of the last assembly's ranks */
  int32_t regrows;          /* compact: assemblies redone after a pool overflow */
  int32_t reserved;
} bem_far_storage;
int bem_get_far_storage(bem_ctx* ctx, bem_far_storage* out);

/* ---- several meshes in one context ------------------------------------------
 * Independent problems (the batched sweep of meshes of uneven size) share one
 * GPU: each added mesh gets its own context state and non-blocking stream,
 * and bem_solve_sweep_batched runs the meshes' sweeps on a pool of up to 16
 * host threads, so the kernels of several meshes share the GPU. The material and
 * window of the context apply to every mesh (set them before the sweep); far
 * storage and pivot reuse settings are taken when the mesh is added. The
 * single-mesh calls (bem_mesh, bem_solve_sweep, ...) keep their own mesh. */
/* Adds a mesh (arguments as bem_mesh) and returns its id 0, 1, ... in
 * *mesh_id. Errors: as bem_mesh. */
int bem_add_mesh(bem_ctx* ctx, const double* xyz, int64_t nv, const int32_t* tri, int64_t ne,
                 const int8_t* bc_type, const bem_opts* opts, int32_t* mesh_id);
/* Number of added meshes (or INVALID_ARG). */
int bem_mesh_count(const bem_ctx* ctx);
/* Sweeps every added mesh with one load history and its own prescribed
 * pattern bc_patterns[id] (ne x 3 each). stats (may be NULL): per mesh id,
 * n_omega / 2 + 1 entries, mesh-major. Returns the first hard error of any
 * mesh, else NOT_CONVERGED if any frequency of any mesh missed the tolerance,
 * else OK; every mesh's results are kept. */
int bem_solve_sweep_batched(bem_ctx* ctx, double T, int32_t n_omega, const double* load_hist,
                            const double* const* bc_patterns, const bem_opts* opts, bem_freq_stats* stats);
/* As bem_get_frequency_solution and bem_time_response, for mesh mesh_id. */
int bem_mesh_frequency_solution(bem_ctx* ctx, int32_t mesh_id, int32_t k, double* out);
int bem_mesh_time_response(bem_ctx* ctx, int32_t mesh_id, const int64_t* dofs, int64_t ndof, double* out);

/* ---- learned initial guess (BEM_GUESS_MLP) ---------------------------------
 * The paper's extrapolation (Sec. 4.2) fits a_k^(0) in the span of the last
 * K solutions. The learned guess adds one candidate column p_k to that span,
 * so its least-squares residual is never above the plain extrapolation's.
 * p_k comes from a pointwise network applied to every unknown d:
 *   x(d) = [Re, Im of a_{k-1..k-4}(d) / S] (8), Re(s_k) dt, Im(s_k) dt,
 *   S = max_d |a_{k-1}(d)|, dt = T / n_omega;
 *   y = W3 tanh(W2 tanh(W1 x + b1) + b2) + b3, p_k(d) = S (y0 + i y1),
 * widths 10 -> 256 -> 256 -> 2. Parameters: one float vector of
 * bem_mlp_num_params() values in the order W1 (256 x 10, row-major), b1 (256),
 * W2 (256 x 256), b2 (256), W3 (2 x 256), b3 (2). The products use the weight
 * matrices rounded to bfloat16 (round to nearest even) with FP32
 * accumulation; biases and the Adam state stay FP32. During a sweep with
 * BEM_GUESS_MLP the network proposes for k >= 4 and, after frequency k is
 * solved, takes `steps` Adam steps (beta 0.9, 0.999, eps 1e-8) on the mean
 * over unknowns of |y - a_k / S|^2 (the two outputs summed). The weights
 * persist in the context across sweeps; without bem_mlp_init or
 * bem_mlp_set_weights they start from a Glorot-uniform draw with seed 3032. */
int64_t bem_mlp_num_params(void);
/* Glorot-uniform weights from `seed`, zero biases, Adam state reset. */
int bem_mlp_init(bem_ctx* ctx, uint64_t seed);
/* Adam steps per solved frequency (>= 0; 0 freezes the weights) and the
 * learning rate (>= 0). Defaults 4 and 1e-3. */
int bem_mlp_set_training(bem_ctx* ctx, int32_t steps_per_frequency, double lr);
/* Copy n = bem_mlp_num_params() host floats in / out; set resets Adam. */
int bem_mlp_set_weights(bem_ctx* ctx, const float* theta, int64_t n);
int bem_mlp_get_weights(bem_ctx* ctx, float* theta, int64_t n);
/* Network outputs y (B x 2) for host features x (B x 10), row-major. */
int bem_mlp_forward(bem_ctx* ctx, const float* x, int64_t B, float* y);
/* Gradient of the loss at host features x (B x 10) and targets t (B x 2)
 * into grad (num_params floats) and the loss into *loss (may be NULL). */
int bem_mlp_gradient(bem_ctx* ctx, const float* x, const float* t, int64_t B, float* grad, double* loss);
/* One Adam step with learning rate lr on that loss (loss before the step). */
int bem_mlp_train_step(bem_ctx* ctx, const float* x, const float* t, int64_t B, double lr, double* loss);

/* ---- measurement ------------------------------------------------------- */

typedef struct bem_profile {
  int64_t hmv_launches;     /* H-matrix products (one launch pair each) */
  double hmv_ms;            /* summed CUDA-event time of those products */
  double hmv_bytes;         /* algorithmic bytes: operator entries used + x read + y written */
  int64_t assemble_calls;   /* operator assemblies */
  double assemble_ms;       /* summed CUDA-event time of assembly (RHS, singular, near, ACA) */
  int64_t kernel_launches;  /* kernels launched by the library since profiling was (re)enabled */
  int64_t aca_blocks;       /* admissible blocks assembled */
  int64_t aca_stepped;      /* of which took ACA steps (were not settled by pivot reuse alone) */
  int64_t aca_failures;     /* admissible blocks of the last assembly whose ACA reached the rank
                               cap (min(3 min(rows, cols), 512)) without meeting aca_tol */
} bem_profile;

/* Enable (1) or disable (0) event timing of the H-matrix products and of
 * assembly on the context's stream, and reset the counters. Timing adds two
 * event records per timed launch; results are complete after any call that
 * synchronises the stream. */
int bem_set_profiling(bem_ctx* ctx, int on);
int bem_get_profile(bem_ctx* ctx, bem_profile* out);

#ifdef __cplusplus
}
#endif

#endif /* BEM_H_ */
