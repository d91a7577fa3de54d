// Kernel launchers provided by the assembly and solver translation units.
#pragma once

#include "bem_internal.h"

namespace bem {

// ---- assembly (bem_assemble.cu) ----
void launch_centroids(const double* xyz, long long nv, const int* tri, int ne, double* cen, double* h,
                      int* bad, cudaStream_t st);
void launch_geometry(const double* xyz, const int* tri, const int* perm, const signed char* bc_in, int ne,
                     ElemF* ef, ElemD* ed, signed char* bc, cudaStream_t st);
void launch_sing_count(const NearBlk* blks, int nblk, const ElemD* ed, int* count, cudaStream_t st);
void launch_sing_fill(const NearBlk* blks, int nblk, const ElemD* ed, const int* offs, SingPair* out,
                      cudaStream_t st);
// Static parts of the singular pairs; fp32: the near-singular rule in FP32
// (enough for the complex64 operator), else FP64.
void launch_static(const SingPair* pairs, int n, const ElemD* ed, const KParams<double>& P, double* out, bool fp32,
                   cudaStream_t st);
void launch_pair_sort(const NearBlk* blks, int nblk, const ElemF* ef, const ElemD* ed, const long long* poff,
                      unsigned* plist, int* pcount, cudaStream_t st);
// Regular near-field entries (near may be null) and, when b is given, the
// near blocks' share of b += pk * B(s) pattern (atomic adds; b zeroed first).
template <typename R, typename Op>
void launch_near_regular(const NearBlk* blks, int nblk, int max_nr, const unsigned* plist, const long long* poff,
                         const int* pcount, const ElemF* ef, const ElemD* ed, const signed char* bc,
                         const KParams<R>& P, Op* near, const float* patf, const double* patd, c128 pk, c128* b,
                         cudaStream_t st);
void launch_polar(const ElemD* ed, int ne, double* out, cudaStream_t st);
template <typename R, typename Op>
void launch_sing(const SingPair* pairs, int n, const ElemD* ed, const double* polar, const signed char* bc,
                 const double* stat, const KParams<R>& P, Op* near, c128* pinv, const double* pattern, c128 pk,
                 c128* b, int* status, cudaStream_t st);
// Far blocks' share of b += pk * B(s) pattern, one warp per row element:
// rng holds (c0, nc) column ranges, rptr the ranges of each leaf, elem_leaf
// the leaf of each element (tree order). Must be the first writer of b after
// it is zeroed (plain read-modify-write per row).
template <typename R>
void launch_rhs_far(const int* rng, const int* rptr, const int* elem_leaf, int ne, const ElemF* ef, const ElemD* ed,
                    const signed char* bc, const float* patf, const double* patd, const KParams<R>& P, c128 pk,
                    c128* b, cudaStream_t st);
// Admissible blocks split in two lists: small ones one warp each, large ones one CTA each.
template <typename R, typename Op>
void launch_aca(const FarBlk* blks, const int* small_list, int nsmall, const int* large_list, int nlarge,
                const ElemF* ef, const ElemD* ed, const signed char* bc, const KParams<R>& P, Op* U, Op* V, int* rank,
                int* fails, double eps, const AcaState& state, cudaStream_t st);
// Reuse of the previous assembly's pivots: evaluates the pivot rows and
// columns at the new s, forms the cross approximation through them and
// writes the start state (kstart, norm0, done) for launch_aca. npiv holds the
// previous pivot counts (rank plus spares); rank and npiv of every block
// settled by the reuse are updated, the others by launch_aca.
// Blocks b0 .. b0 + nfar - 1.
template <typename R, typename Op>
cudaError_t launch_aca_warm(const FarBlk* blks, int b0, int nfar, const ElemF* ef, const ElemD* ed,
                            const signed char* bc, const KParams<R>& P, Op* U, Op* V, int* rank, int* npiv,
                            int* piv_i, int* piv_j, int* kstart, double* norm0, int* done, double eps, double tau,
                            cudaStream_t st);
// Factor offsets of full storage: fbase[2b], fbase[2b + 1] = uoff, voff.
void launch_fbase_full(const FarBlk* blks, int nfar, long long* fbase, cudaStream_t st);
// Compact storage: packs blocks b0 .. b0 + nblk - 1 from the workspace (wsU,
// wsV at the blocks' uoff, voff) at their ranks into the pools U, V of
// capU, capV entries, taking space from cursor[0], cursor[1]; writes fbase.
template <typename Op>
void launch_far_pack(const FarBlk* blks, int b0, int nblk, const int* rank, const Op* wsU, const Op* wsV, Op* U,
                     Op* V, long long capU, long long capV, long long* fbase, unsigned long long* cursor,
                     cudaStream_t st);

// ---- solver (bem_solve.cu) ----
// H-matrix product y = A x for nrhs right-hand sides (x, y: nrhs vectors of
// length N, stride N). Op: operator storage; X: input vectors; Y: output;
// accumulation in Acc (float or double).
// run (optional): the launch does nothing unless *run is nonzero.
template <typename Op, typename X, typename Y, typename Acc>
void launch_hmatvec(const bem_ctx* ctx, const Op* near, const Op* U, const Op* V, cplx<Acc>* t,
                    const X* x, Y* y, int nrhs, cudaStream_t st, const int* run = nullptr);

// y = A x (c64 operator, FP32 accumulation, one right-hand side) with
// caller-provided scratch: t (t_entries values) and part (part_rows values).
void launch_hmatvec_scratch_c64(const bem_ctx* ctx, const c64* near, const c64* U, const c64* V, cplx<float>* t,
                                cplx<float>* part, const c64* x, c64* y, cudaStream_t st);

// z = M^{-1} v per element (3x3 inverse diagonal blocks); run (optional): the
// launch does nothing unless *run; joff (optional): v taken at v + (*joff) ldv
template <typename Pm, typename V, typename Z>
void launch_precond(const Pm* pinv, const V* v, Z* z, int ne, cudaStream_t st, const int* run = nullptr,
                    const int* joff = nullptr, long long ldv = 0);

// Partial dot products part[l * nblk + blk] of conj(V_l) . w, l < nvec (FP64)
template <typename Vb, typename W>
int launch_dots(const Vb* V, long long ldv, int nvec, const W* w, long long n, c128* part, cudaStream_t st);
// One Arnoldi orthogonalisation step (CGS2 against V_0..V_j, norm, and
// V_{j+1} = w / ||w||) in a single cooperative launch; hcol receives
// [h1 (m+1) | h2 (m+1) | ||w||^2]; part needs (2 (j+1) + 1) x
// arnoldi_orth_max_blocks() complex values.
// With gm (the device-driven solver): j and the column slot come from its
// state, the launch does nothing outside a cycle, and the step's Givens
// rotation and convergence test are taken on the device (bem_solve.cu).
template <typename Vb>
cudaError_t launch_arnoldi_orth(Vb* V, long long ldv, int j, Vb* w, long long n, c128* part, c128* hcol, int m,
                                cudaStream_t st, const GmDev* gm = nullptr);
// Device-driven GMRES: start of a solve (bb: ||b||^2 on the device), the
// true-residual test that ends the solve or starts a cycle (rr: ||r||^2;
// V0 = r / ||r||), and the update out = V R^{-1} g that closes a cycle.
void launch_gm_init(const GmDev& d, const c128* bb, cudaStream_t st);
template <typename Vb>
void launch_gm_begin(const GmDev& d, const c128* rr, const c128* r, Vb* V0, c128* x, long long n, cudaStream_t st);
template <typename Vb>
void launch_gm_combine(const Vb* V, long long ldv, const GmDev& d, c128* out, long long n, cudaStream_t st);
int arnoldi_orth_max_blocks();
// Solution extrapolation fit (Sec. 4.2) after Y = A X (C columns of n, c128):
// CGS2 QR, s = R^{-1} Q^H b, a0 = X s, and the residual estimates res[0..1]
// (device), in one cooperative launch. Q: C x n scratch; part: 3 (SEM_MAXC + 1)
// x arnoldi_orth_max_blocks() complex values.
constexpr int SEM_MAXC = 5;
cudaError_t launch_sem_fit(const c128* const* X, int C, int K, const c128* Y, const c128* b, c128* Q, c128* part,
                           c128* a0, double* res, long long n, cudaStream_t st);
// out[l] = sum_blk part[l * nblk + blk]
void launch_dots_final(const c128* part, int nblk, int nvec, c128* out, cudaStream_t st);
// r = b - y ; both c128
void launch_residual(const c128* b, const c128* y, c128* r, long long n, cudaStream_t st);
void launch_axpy(c128 a, const c128* x, c128* y, long long n, cudaStream_t st, const int* run = nullptr);
void launch_copy_cast(const c128* x, c64* y, long long n, double scale, cudaStream_t st);
void launch_copy_cast(const c128* x, c128* y, long long n, double scale, cudaStream_t st);

// Eq. DFT-MFT for k = 0..n_omega/2
void launch_load_dft(const double* P, int n_omega, double T, double eta, c128* out, cudaStream_t st);
// Eq. IDFT-MFT: spec (nf x ldspec, columns at dof indices idx or 0..ndof-1)
void launch_idft(const c128* spec, long long ldspec, const long long* idx, long long ndof, int n_omega,
                 double T, double eta, int window, double* out, cudaStream_t st);

// ---- interior field (bem_interior.cu) ----
// Displacement at npts interior points (caller coordinates, FP64) from the
// boundary solution a (tree order) and the prescribed pattern * pk.
template <typename R>
void launch_interior(const double* pts, int npts, const ElemD* ed, int ne, const signed char* bc, const c128* a,
                     const double* pattern, c128 pk, const KParams<R>& P, c128* out, cudaStream_t st);
// The six points x +- h e_a around each point, and the strain from the
// displacements there (central differences; npts x 6 complex).
void launch_offset_points(const double* pts, int npts, double h, double* out, cudaStream_t st);
void launch_strain(const c128* uoff, int npts, double h, c128* eps, cudaStream_t st);

// ---- leaf-block preconditioner (bem_precond.cu) ----
// Inverses of the leaves' diagonal blocks of the near storage (FP32 Gauss-
// Jordan for complex64 blocks, FP64 for complex128); pinv3: the 3 x 3 block
// inverses a leaf falls back to if its block is singular.
template <typename R>
cudaError_t launch_leaf_inverse(const LeafPre* leaves, int nleaves, const cplx<R>* near, const c128* pinv3,
                                cplx<R>* out, cudaStream_t st);
// z = M^-1 v with the leaf inverses (tree order vectors)
template <typename Pm, typename V, typename Z>
void launch_leaf_apply(const LeafPre* leaves, int nleaves, const Pm* minv, const V* v, Z* z, cudaStream_t st,
                       const int* run = nullptr, const int* joff = nullptr, long long ldv = 0);

}  // namespace bem
