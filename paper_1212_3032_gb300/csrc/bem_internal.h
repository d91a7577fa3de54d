// Internal declarations shared by the library's translation units: device
// data layouts of the mesh and of the hierarchical operator, the context,
// and the kernel launchers each unit provides.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "bem_common.cuh"
#include "bem_tree.h"

namespace bem {

// ---- device element geometry (tree order) --------------------------------
// FP32 view: centroid split into hi + lo floats (so centroid differences are
// accurate in FP32), vertex p0 relative to the centroid, edges, normal.
struct ElemF {
  float c_hi[3], c_lo[3];
  float o0[3], e1[3], e2[3];
  float n[3];
  float area2;  // 2 * area
  float h2;     // (longest edge)^2
};
// FP64 view for the singular / near-singular rules.
struct ElemD {
  double c[3];
  double p0[3], p1[3], p2[3];
  double n[3];
  double area2;
  double h2;
};

// Dense near-field block (tau rows x sigma cols), column-major with the
// leading dimension ld = 3 nr rounded up to even and an even offset (16-byte
// aligned columns); the padding row is zero.
struct NearBlk {
  long long off;  // offset in the near-field array (entries, even)
  int r0, nr;     // row cluster: first tree element, element count
  int c0, nc;     // column cluster
  int ld;         // leading dimension (even, >= 3 nr)
};

// Rank cap of the admissible blocks: rmax = min(3 min(nr, nc), ACA_RANK_CAP).
constexpr int ACA_RANK_CAP = 512;
// Compact storage: the pools start at every block's factors at this rank (or
// its cap if lower) and grow on demand.
constexpr int POOL_INIT_RANK = 20;

// Low-rank far-field block A ~ U V^T; U: (3 nr) x rmax column-major,
// V: (3 nc) x rmax column-major; rank[b] <= rmax set by ACA.
struct FarBlk {
  long long uoff, voff;  // this block's U, V while ACA runs: offsets in the U, V arrays it
                         // writes (the stored factors in full storage; the workspace of
                         // the block's batch in compact storage)
  int r0, nr, c0, nc;
  int rmax;
  int toff;  // offset of this block's t = V^T x in the t buffer
  int flat;  // one of its clusters is faceted (flat faces: most elements share a few normals)
};

// One column panel of a leaf row of the matrix-vector product:
// y[rows of leaf] += P x_panel, P column-major with leading dimension ld.
struct Panel {
  long long data;  // offset into the near array (kind 0); kind 1: row offset within the
                   // block's U (its start comes from the operator set's factor offsets)
  int ld;          // leading dimension of the stored block
  int ncols;       // kind 0: columns; kind 1: ignored (rank read at run time)
  int xoff;        // kind 0: first x index; kind 1: far block index
  int kind;
};

// A contiguous run of panels of one leaf row handled by one CTA of the
// matrix-vector product; its partial row sums go to rows [slot, slot + rows)
// of the partial buffer and are added up per leaf in a fixed order.
struct Task {
  int leaf;
  int p0, p1;  // panel range (all near panels, or all far panels)
  int slot;
  int kind;    // 0: near panels, 1: far panels
};

// One leaf's diagonal block for the leaf-block preconditioner: the near
// block of the leaf with itself (offset, leading dimension, m = 3 nr rows),
// the leaf's first element (tree order) and its inverse's place (column-major,
// leading dimension ldo, even).
constexpr int LEAF_PRE_MAX_ELEMS = 64;
struct LeafPre {
  long long off;
  long long ooff;
  int ld, m, ldo, e0;
};

// Work item of the fused H-matrix product (one CTA each): kind 0 = the
// dense near panels [p0, p1) of leaf l0 (a near Task's panels); kind 1 = the
// admissible blocks far_list[p0, p1), all with the same row cluster (t = V^T x
// for each, then sum_b U_b t_b over the row cluster, leaves [l0, l1)). Its
// rows go to the partial buffer from row `slot` on.
struct HItem {
  long long slot;
  int kind;
  int p0, p1;  // kind 1: a range of the far-block list (blocks of one row cluster)
  int l0, l1;
};
constexpr int HITEM_MAX_BLOCKS = 24;    // admissible blocks per far item
constexpr int HITEM_MAX_TCOLS = 2048;   // their rank caps summed (V^T x values kept in shared memory)

// Singular (SELF) and near-singular (NEAR) element pairs, FP64 path.
struct SingPair {
  int i, e;         // collocation element, integration element (tree order)
  long long entry;  // near-array offset of entry (row 3 i', col 3 e')
  int ld;           // leading dimension of that block
  int self;         // 1 for i == e
};

// Start state of the ACA kernels (cross-frequency pivot reuse). Pivots are
// recorded for every block at offset FarBlk::toff; kstart / norm0 / done may
// be null (every block starts from rank 0).
constexpr int WARM_RMAX = 128;  // largest reused rank (blocks above restart ACA at every frequency)
constexpr int WARM_SPLIT = 64;  // rank classes of the reuse solve: (0, 64] and above
struct AcaState {
  const int* kstart;    // per far block: rank to continue from
  const double* norm0;  // per far block: ||S||_F^2 estimate at that rank
  int* done;            // per far block: 1 = converged already (skip); 2 = converged on the
                        // reused pivots, check rows pending (set to 1 or 0 by the ACA kernels)
  int* piv_i;           // pivot row of each step (block-local scalar index)
  int* piv_j;           // pivot column of each step
  int* npiv;            // per far block: pivots recorded (rank plus spares)
};

template <typename T> struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  cudaError_t alloc(size_t count) {
    release();
    if (count == 0) return cudaSuccess;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e == cudaSuccess) n = count;
    else p = nullptr;
    return e;
  }
  cudaError_t ensure(size_t count) { return count <= n ? cudaSuccess : alloc(count); }
};

// Process-wide count of kernel launches issued by the library (for the
// launch count reported by measurements). count_if(c) adds one when c holds.
bool count_if(bool c);
long long launch_count();

// Device-side state of one GMRES solve (restarted GMRES, right
// preconditioning, Sec. 3.1). The kernels of an Arnoldi step, of the update
// that closes a cycle and of the true-residual test read and advance it, so
// that the host enqueues a solve's work without waiting on any step. The
// kernels that change it also write a copy to mapped host memory, from which
// the host learns, a few steps later, that a cycle or the solve has ended.
constexpr int GM_MAX_CYCLES = 256;  // cycles whose step counts are recorded
struct GmCtl {
  int active;     // a cycle is under way: the step kernels do their work
  int j;          // Arnoldi steps taken in the current cycle
  int update;     // the cycle has ended; the update of x is pending
  int live;       // the solve has not finished
  int its;        // Arnoldi steps over all cycles
  int cycles;     // cycles started
  int converged;  // the true residual met the tolerance
  int arrive;     // blocks of the residual test that have read the state
  double bnorm, rel, guess_rel, target;
  int jdone[GM_MAX_CYCLES];  // steps taken by each cycle
};
// What the device-driven kernels share (passed by value).
struct GmDev {
  GmCtl* ctl;          // device state
  GmCtl* mirror;       // its mapped host copy (device address)
  c128* R;             // rotated Hessenberg columns: column j at R + j (m + 1)
  c128* g;             // m + 1: rotated right-hand side of the small least-squares problem
  c128* cs;            // m: Givens rotations (cosines)
  c128* sn;            // m: (sines)
  c128* hcol;          // the steps' Hessenberg column slots, slot_len apart
  long long slot_len;
  int m, max_iters;
  double tol;          // on ||r|| / ||b||
  double floor;        // inner target relative to the cycle's first residual
};

struct MlpState;  // learned initial guess (bem_mlp.cu)

// The storage of one assembled operator and its right-hand side. A sweep
// keeps up to three: frequencies k + 1 and k + 2 are assembled into the
// others while GMRES runs on the set of frequency k (the context's fields
// hold the set in use; swap_ops exchanges it with one of the others).
struct OpSet {
  DevBuf<c64> near32, u32, v32, prec_inv32, minv32;
  DevBuf<c128> near64, u64, v64, prec_inv, b64, minv64;
  DevBuf<int> rank, aca_fail, status;
  DevBuf<long long> fbase;
  bool near_zero_pending = true;
  bool minv_ready = false;
  bool fbase_ready = false;
  int prof_slot = 0;
};

// A run of consecutive admissible blocks whose ACA factors, at their rank
// caps, fit the workspace together (compact storage); full storage has one
// batch over all blocks. The size-class lists hold each batch's blocks in
// the index ranges [s0, s1) and [l0, l1).
struct FarBatch {
  int b0, b1;
  int s0, s1, l0, l1;
};

// Host-side rule tables (Gauss-Legendre on [0,1], series coefficients).
void make_rule_tables(RuleTables& t);

// Translation-unit uploads of the constant tables.
cudaError_t upload_rules_assemble(const RuleTables& t, cudaStream_t st);
cudaError_t upload_rules_interior(const RuleTables& t, cudaStream_t st);

}  // namespace bem

struct bem_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;

  // material (Sec. 2.1)
  bool have_mat = false;
  double E = 0, nu = 0, rho = 0, mu = 0, lam = 0, cs = 0, cp = 0;
  // window (Sec. 3)
  double eta = 0;
  int window = BEM_WIN_NONE;

  // mesh
  bool have_mesh = false;
  int ne = 0;
  long long N = 0;
  bem_opts mesh_opts{};
  bem::ClusterTree tree;
  std::vector<signed char> bc_host;  // tree order
  bem::DevBuf<bem::ElemF> ef;
  bem::DevBuf<bem::ElemD> ed;
  bem::DevBuf<signed char> bc;       // tree order
  bem::DevBuf<int> perm;             // tree -> caller
  bem::DevBuf<int> iperm;            // caller -> tree

  // operator structure (frequency independent)
  std::vector<bem::NearBlk> near_h;
  std::vector<bem::FarBlk> far_h;
  bem::DevBuf<bem::NearBlk> near_d;
  bem::DevBuf<bem::FarBlk> far_d;
  long long near_entries = 0, u_entries = 0, v_entries = 0;  // u/v: factors at their rank caps
  long long u_init = 0, v_init = 0;   // compact pools' first size (entries)
  int t_entries = 0;
  // far-field factor storage (bem_set_far_storage): full = every block at its
  // rank cap, written in place by ACA; compact = ACA runs batch by batch in a
  // workspace and each batch is packed at its actual ranks into pools that
  // grow on demand
  int far_mode_req = BEM_FAR_AUTO;
  long long far_ws_req = 0;            // requested workspace bytes (0: default)
  bool far_compact = false;            // storage chosen for the current mesh
  std::vector<bem::FarBatch> far_batches;
  long long ws_entries = 0;            // workspace entries per factor (U half, V half)
  int far_regrows = 0;                 // pool regrowths (assemblies re-run after an overflow)
  // compact storage in a pipelined sweep: the pools' need of the assembly
  // made on the assembly stream is read (and an overflow redone) only when
  // its operator set comes into use, so that the host does not wait for it
  bool far_defer = false;              // set around such an assembly
  double mem_share = 1.0;              // share of the free device memory a second operator set may take (batch: 1 / meshes)
  bool far_verify_pending = false;
  double far_pending_s[2] = {0, 0};    // its s (re, im)
  cudaEvent_t ev_far_cursor = nullptr;
  bool far_was_ok = false;             // the current assembly started from stored pivots
  bem::DevBuf<bem::c64> ws32;          // 2 x ws_entries
  bem::DevBuf<bem::c128> ws64;
  int nleaves = 0;
  std::vector<int> leaf_nodes;        // node index per leaf (row order)
  bem::DevBuf<int> leaf_r0, leaf_nr;  // per leaf
  bem::DevBuf<int> panel_ptr;         // CSR over leaves
  bem::DevBuf<bem::Panel> panels;
  int ntasks = 0;
  long long part_rows = 0;            // rows of the partial buffer per right-hand side
  bem::DevBuf<bem::Task> tasks;
  bem::DevBuf<int> task_order;        // task indices by size, largest first (launch order)
  // fused product: items in launch order (largest estimated cost first), and
  // per leaf the partial-buffer offsets of its rows in each contribution
  int nhitems = 0;
  long long hpart_rows = 0;           // rows of the partial buffer per right-hand side
  bem::DevBuf<bem::HItem> hitems;
  bem::DevBuf<int> hfar_list;         // admissible blocks grouped by row cluster (far items' ranges)
  int hitem_tcols = 0;                // largest sum of rank caps over a far item
  bem::DevBuf<int> hc_ptr;            // CSR over leaves
  bem::DevBuf<long long> hc_off;
  cudaStream_t aux_stream = nullptr;  // the far-field assembly runs here, joined back to stream
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaStream_t asm_stream = nullptr;  // a sweep assembles frequency k + 1 here while GMRES(k) runs
  cudaEvent_t ev_asm_ring[3] = {};    // a sweep's assembly of frequency f has completed (slot f mod depth)
  // a sweep runs the caller's part of its work (guess, GMRES, IDFT) on this
  // stream of the device's greatest priority, so that blocks of the
  // overlapped assembly (least priority) do not delay it; joined to `stream`
  cudaStream_t solve_stream = nullptr;
  cudaEvent_t ev_solve_in = nullptr, ev_solve_out = nullptr;
  bem::OpSet back[2];                 // the operator sets not in use (see swap_ops)
  bem::DevBuf<int> leaf_cnt;          // per leaf: tasks completed in the current product (reset to 0 after it)
  bem::DevBuf<int> task_ptr;          // CSR of tasks over leaves
  bem::DevBuf<double> part;           // partial sums (sized for 4 rhs of complex FP64)
  int max_nr = 0;                     // largest leaf (elements)
  bem::DevBuf<long long> poff;        // per near block: offset of its sorted pair list
  bem::DevBuf<unsigned> plist;        // sorted regular pairs of the near blocks
  bem::DevBuf<int> pcount;            // regular pairs per near block
  bem::DevBuf<int> rhs_rng;           // far RHS: (c0, nc) column ranges of each leaf's far panels
  bem::DevBuf<int> rhs_rptr;          // CSR of those ranges over leaves
  bem::DevBuf<int> elem_leaf;         // leaf of each element (tree order)
  bem::DevBuf<float> patf;            // prescribed pattern (tree order, FP32)
  int nfar_small = 0, nfar_large = 0;
  bem::DevBuf<int> far_small, far_large;  // admissible block indices by size class
  bem::DevBuf<double> polar;          // ne x 27 self-rule polar parameters
  // singular pairs and their static parts
  int nsing = 0;
  bem::DevBuf<bem::SingPair> sing;
  bem::DevBuf<double> sing_static;    // nsing x 18 (U* 9, T* 9)
  bool static_fp64 = false;           // sing_static from the FP64 near-singular rule
  bem::DevBuf<int> loaded;            // tree elements with nonzero prescribed pattern
  int nloaded = 0;

  // operator values at the current frequency
  int prec = BEM_PREC_C64_MIXED;
  bool assembled = false;
  double s_re = 0, s_im = 0;
  bool near_zero_pending = true;       // zero the near storage once after (re)allocation (padding rows)
  bem::DevBuf<bem::c64> near32, u32, v32, t32;
  bem::DevBuf<bem::c128> near64, u64, v64, t64;
  bem::DevBuf<int> rank;
  bem::DevBuf<int> aca_fail;
  // per admissible block: offsets of its stored U and V ([2b], [2b + 1]);
  // then the pool cursors (entries the last assembly needed)
  bem::DevBuf<long long> fbase;
  bool fbase_ready = false;            // full storage: offsets filled for this set
  // cross-frequency reuse of ACA pivots
  bool aca_reuse = true;               // bem_set_aca_reuse
  bool aca_warm_ok = false;            // pivots of a previous assembly of this mesh are stored
  bool aca_last_warm = false;          // the last assembly started from reused pivots
  double aca_tau = 0.1;                // pivot test of the reused steps
  bem::DevBuf<int> piv_i, piv_j;       // t_entries each
  bem::DevBuf<int> piv_snap;           // compact storage: piv_i, piv_j, npiv an assembly started from
  bem::DevBuf<int> aca_kstart, aca_done, aca_npiv;
  bem::DevBuf<double> aca_norm0;
  long long prof_aca_blocks = 0;       // far blocks assembled (profiling)
  long long prof_aca_continued = 0;    // of which took ACA steps (not settled by reuse alone)
  bem::DevBuf<int> status;             // singular 3x3 diagonal block flag
  bem::DevBuf<bem::c128> prec_inv;     // ne x 9 inverse diagonal blocks
  bem::DevBuf<bem::c64> prec_inv32;
  // leaf-block preconditioner (BEM_PRECOND_LEAF): the leaves' diagonal blocks,
  // their inverses at the current frequency, and which preconditioner the
  // solves use (a sweep with BEM_PRECOND_AUTO decides at its first k > 0)
  int nleaf_pre = 0;                   // 0: leaves above LEAF_PRE_MAX_ELEMS (unavailable)
  long long leaf_pre_entries = 0;
  bem::DevBuf<bem::LeafPre> leaf_pre;
  bem::DevBuf<bem::c64> minv32;
  bem::DevBuf<bem::c128> minv64;
  bool minv_ready = false;             // inverses of the set in use match its operator
  bool use_leaf_pre = false;           // the solves apply the leaf inverses
  int pre_auto = 0;                    // BEM_PRECOND_AUTO in a sweep: 0 undecided, 1 3x3 kept, 2 leaf kept

  // solver workspace
  bem::DevBuf<bem::c64> V32;           // Krylov basis (m+1) x N
  bem::DevBuf<bem::c128> V64;
  bem::DevBuf<bem::c64> w32;
  bem::DevBuf<bem::c128> w64, x64, r64, b64, y64, tmp64;
  bem::DevBuf<double> red;             // reduction scratch
  bem::DevBuf<bem::c128> orth_part;    // partial sums of the Arnoldi orthogonalisation step
  bem::DevBuf<double> pattern;         // tree order ne x 3
  double* host_red = nullptr;          // pinned
  std::vector<cudaEvent_t> col_events; // one per Arnoldi step of a cycle (the host reads the solver state after them)
  bem::DevBuf<bem::GmCtl> gm_ctl;      // device-driven GMRES: state
  bem::GmCtl* gm_mirror = nullptr;     // its mapped host copy (host address)
  bem::GmCtl* gm_mirror_dev = nullptr; // (device address)
  bem::DevBuf<bem::c128> gm_work;      // rotated columns, g, cs, sn
  bem::DevBuf<bem::c64> gm_w32, gm_z32;   // product output and preconditioned input of a step
  bem::DevBuf<bem::c128> gm_w64, gm_z64;
  cudaEvent_t ev_free_ring[3] = {};   // a sweep's solve of frequency f has completed (its set is free)
  double* sweep_pin = nullptr;         // pinned per-frequency results of a sweep (extrapolation residuals,
  size_t sweep_pin_n = 0;              // ACA failure counts), read after it

  // event timing (bem_set_profiling)
  bool profiling = false;
  struct Pending {
    cudaEvent_t a, b;
    double base, mult;  // bytes = base + mult x (low-rank entries in use at slot)
    int slot;           // assembly slot of prof_dev holding those entries (0: none)
    int kind;           // 0 H-matrix product, 1 assembly
  };
  std::vector<Pending> pending;
  // profiling counters kept on the device, so that profiling adds no host
  // synchronisation: prof_dev[0] = blocks that took ACA steps after reuse,
  // prof_dev[s] (s >= 1) = low-rank entries in use after the s-th assembly
  bem::DevBuf<long long> prof_dev;
  int prof_slot = 0, prof_nslots = 0;
  struct DoneProduct {
    double base, mult;
    int slot;
  };
  std::vector<DoneProduct> prof_products;  // timed products awaiting their byte counts
  std::vector<cudaEvent_t> event_pool;
  long long prof_hmv_launches = 0, prof_asm_calls = 0;
  long long launches_at_reset = 0;  // library kernel launches counted when profiling was (re)enabled
  double prof_hmv_ms = 0, prof_asm_ms = 0;

  // learned initial guess
  bem::MlpState* mlp = nullptr;
  int mlp_steps = 4;       // Adam steps after each solved frequency
  double mlp_lr = 1e-3;
  bem::DevBuf<bem::c128> sem_work;     // extrapolation workspace (3 x columns x N)
  bem::DevBuf<bem::c128> sem_part;     // its partial sums
  bem::DevBuf<double> sem_res;         // its residual estimates

  // several meshes in one context (bem_add_mesh): each in a child context
  // with its own non-blocking stream; the children's cooperative launches
  // share one stream (CoopLane)
  std::vector<bem_ctx*> batch;
  cudaStream_t batch_coop = nullptr;   // the children's shared stream (owned by the parent)
  cudaStream_t coop_stream = nullptr;  // in a child: the parent's batch_coop (borrowed)
  cudaEvent_t coop_in = nullptr, coop_out = nullptr;

  // sweep results
  int n_omega = 0;
  double T = 0;
  int nf = 0;
  bem::DevBuf<bem::c128> sol;          // nf x N (tree order)
  bem::DevBuf<bem::c128> Pk;           // nf
  std::vector<bem::c128> Pk_host;
};

namespace bem {
int fail(bem_ctx* ctx, int code, const std::string& msg);
// learned initial guess (bem_mlp.cu)
void mlp_free(bem_ctx* ctx);
int mlp_ready(bem_ctx* ctx);
int mlp_propose(bem_ctx* ctx, const c128* const* prev, double sre_dt, double sim_dt, const c128** out);
int mlp_train(bem_ctx* ctx, const c128* const* prev, const c128* ak, double sre_dt, double sim_dt, int steps,
              double lr);
int fail_cuda(bem_ctx* ctx, cudaError_t e, const char* what, const char* file, int line);
}
