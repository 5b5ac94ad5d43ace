// Internal declarations shared by the host code (api.cpp, factor_host.cpp) and
// the device code (kernels.cu).  Not part of the public ABI.
#pragma once

#include <array>
#include <cstddef>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/smpc.h"

namespace smpc {

void set_error(const char* fmt, ...);

// ---------------------------------------------------------------------------
// Host FP64 dense linear algebra for the factor step (App. A, App. B).
struct HostFactor {
  int n_x = 0, n_u = 0, n_d = 0, n_e = 0, n_v = 0;
  std::vector<double> L;      // n_u x n_v, orthonormal basis of null(E)
  std::vector<double> Bbar;   // n_x x n_v
  std::vector<double> Rhat;   // n_u x n_v
  std::vector<double> Rbar;   // n_v x n_v
  std::vector<double> Lam;    // n_v x n_v, -Rbar^{-1}
  std::vector<double> Pu;     // n_u x n_d, u_hat(d) = Pu d (minimum-norm particular solution)
  std::vector<double> Pe;     // n_x x n_d, e(d) = B u_hat(d) + Gd d
  std::vector<double> diagB;  // n_x, diag(Bbar Rbar^{-1} Bbar')
  std::vector<double> diagL;  // n_u, diag(L Rbar^{-1} L')
};
// Returns SMPC_OK or SMPC_EINVAL (rank-deficient E, W_u not positive definite).
int host_factor(const smpc_network& net, const double* W_u, HostFactor& out);

// ---------------------------------------------------------------------------
// Tree structure after validation (host copy + device mirrors).
// Forward-sweep segment b (top nodes first, then chains), kSegInts ints:
// {par, path begin, path length, tree, chain begin, chain length, 0, 0}.  par is the
// top node itself for a top segment (chain length 0) and the top node above the
// chain head for a chain (-1 when the chain starts at a root).
constexpr int kSegInts = 8;

struct DevTree {
  int* parent = nullptr;
  int* stage = nullptr;
  int* child_begin = nullptr;
  int* child_count = nullptr;
  int* chain_off = nullptr;     // n_chains + 1
  int* chain_node = nullptr;    // chain nodes, top-down
  int* chain_parent = nullptr;  // top node above each chain head, or -1
  int* top_nodes = nullptr;     // n_top
  int* top_expect = nullptr;    // per node: arrivals a top node waits for (children + 1)
  int* path_off = nullptr;      // per node (n + 1): path of a top node, root .. node
  int* path_node = nullptr;
  int* tree_of = nullptr;       // per node: its tree (the index of its root)
  int* row = nullptr;           // per node: its row of the stage-indexed step data
  int* seg = nullptr;           // kSegInts per forward-sweep segment (top nodes, then chains)
  double* prob = nullptr;
  double* pbar = nullptr;       // p_n + sum of children's p (App. A)
};

}  // namespace smpc

struct smpc_tree {
  int n = 0, N = 0, n_leaves = 0, max_chain_len = 0, device = 0;
  int R = 1;     // trees (roots are nodes 0 .. R-1)
  int rows = 0;  // rows of stage-indexed step data: the sum of the trees' horizons
  std::vector<int> tree_of, row, row_off;
  std::vector<int> parent, stage, child_begin, child_count;
  std::vector<double> prob, pbar;
  std::vector<int> chain_off, chain_node, chain_parent;
  std::vector<int> top_nodes, is_top, top_expect;
  std::vector<int> path_off, path_node;
  std::vector<int> seg;  // forward-sweep segment descriptors (kSegInts each)
  smpc::DevTree dev;
};

namespace smpc {

// Device-side parameters of the iteration kernel.  VT: vector type, MT: matrix type.
struct IterArgs {
  int n, n_x, n_u, n_v, n_k;     // n_k = n_x + n_u rows of [Bbar; L]
  int n_chains, n_top;
  const int* parent;
  const int* child_begin;
  const int* child_count;
  const int* chain_off;
  const int* chain_node;
  const int* chain_parent;
  const int* top_nodes;
  const int* top_expect;
  const int* path_off;
  const int* path_node;
  const int* tree_of;            // per node: its tree (p0 has one state per tree)
  const int* seg;                // kSegInts per forward-sweep segment, 32-byte aligned
  const void* packs;             // per node: [Bbar; L] (n_k x n_v) then Lambda/(2 p_n) (n_v x n_v)
  long long pack_stride;         // entries between consecutive nodes' packs (0: one shared pack)
  const void* pscale;            // shared pack: per node 1 / (2 p_n), applied to Lambda r; else NULL
  void* ybuf0;                   // y^k for even k: n x (2 n_x + n_u) of the state type
  void* ybuf1;                   // y^k for odd k (float64, or float32 pairs hi + lo)
  void* wbuf;                    // w^nu restricted to (xi, psi): n x n_k
  void* h;                       // [Bbar delta; L delta]: n x n_k (anchored: the part on w - w_a)
  void* ha;                      // anchored solves: h at the anchor w_a (n x n_k), else NULL
  void* wa;                      // anchored solves: the anchor w_a (n x n_k)
  const void* uhat;              // n x n_u
  const void* e;                 // n x n_x
  const void* beta;              // n x n_v
  void* spub;                    // n x n_x  (published s of chain heads / top nodes)
  void* rpub;                    // n x n_v
  void* uout;                    // n x n_u
  void* xout;                    // n x n_x
  const void* step_s;            // n
  const void* step_z;            // n
  const void* step_p;            // n x n_u
  const void* inv_s;             // n: 1 / step_s
  const void* inv_z;             // n: 1 / step_z
  const void* inv_p;             // n x n_u: 1 / step_p
  const void* mu_s;              // n: weight mu_S,n of the safety distance block
  const void* x_s;
  const void* x_min;
  const void* x_max;
  const void* u_min;
  const void* u_max;
  const void* p0;                // n_x measured state
  const void* A;                 // n_x x n_x dynamics matrix (row-major), or NULL for A = I
  double gamma_d;
  const double* cvec;            // extrapolation coefficients c_nu, nu = 0..max_iters
  const double* theta;           // theta_nu, nu = 0..max_iters (the ergodic average's weights)
  void* xbar;                    // ergodic average of x (n x n_x), or NULL (not kept)
  void* ubar;                    // ergodic average of u (n x n_u), or NULL
  unsigned long long* res;       // per iteration: rho, ||Hz||, ||t|| as float64 bits
  int* counters;                 // per node arrival counters (top nodes)
  int* flags;                    // [0] iterations done (-1 running), [1] error code
  double tol;
  double* pw;                    // power iteration: [k] ||y_k||^2, [K + k] <y_k, y_{k+1}>
  int pw_len;
  unsigned long long wait_ns;    // bound of the per-node pack pipeline waits of node_mv
  // Forests (R > 1 trees): each tree stops at its own first iterate whose relative residual
  // meets tol.  res_tree: per iteration and tree, (rho, ||Hz||, ||t||) as float64 bits, or
  // NULL (one residual for the whole forest); tree_done: per tree, the iterations it ran
  // once it stopped, -1 while it runs (NULL: none).
  int R;
  unsigned long long* res_tree;
  int* tree_done;
  // Shards of a tree split over several GPUs: the nodes this GPU updates in the prox
  // (its chains and the replicated top nodes), or NULL for all n nodes.
  const int* node_list;
  int n_list;
};

enum KernelMode : int {
  MODE_PROX = 1,      // forward of iteration nu-1, prox, dual update (Phase P)
  MODE_BWD = 2,       // backward sweep of iteration nu
  MODE_LINEAR = 4,    // power iteration on the (scaled) dual Hessian: no affine data, no prox
  MODE_CHECK = 8,     // honour the stop flag / tolerance
  MODE_ANCHOR = 16,   // anchored solve: evaluate the whole solve step at w_a = w^nu into ha
  MODE_DELTA = 32,    // anchored solve: solve step on w^nu - w_a, without the affine data
  MODE_GT = 64,       // backward sweep up to r only: s, g = [Bbar; L]'[s; psi], r for every node
  MODE_WREADY = 128,  // w^nu was written by an earlier launch of the iteration
  MODE_NOCLIMB = 256,  // chain pass of a shard: chains publish their heads' s and r, no top-node climb
  MODE_WONLY = 512     // prox launch writes w^nu of an iteration without a prox (as with MODE_BWD) while
                       // the backward sweep is launched separately
};

enum Schedule : int {
  SCHED_CHAIN = 1,   // one apg_iter launch per iteration, one CTA per chain
  SCHED_NODE = 2,    // six launches per iteration, one task per node in each
  SCHED_HYBRID = 3,  // node-parallel forward sweep and prox, a chain pass up to r, node-parallel Lambda / [Bbar; L]
  SCHED_FUSED = 4    // node-parallel forward sweep and prox, then the whole backward sweep as one chain pass
};
constexpr int kSchedules = 4;

struct LaunchCfg {
  int schedule = SCHED_CHAIN;
  int grid = 1, block = 256;
  size_t smem = 0;
  int stages = 1;           // chain schedule: pack slots per CTA (0: does not fit)
  // node schedule
  int grid_prox = 1, grid_scan = 1, grid_mv = 1, grid_fwd = 1;
  size_t smem_prox = 0, smem_gt = 0, smem_dh = 0;
  size_t smem_fwd = 0;   // forward sweep: staged node vectors
  size_t smem_pstage = 0;  // prox: smem_prox plus the per-warp staging of the node data
  int s_gt = 0, s_dh = 0;   // pack slots of the two mat-vec launches (0: does not fit)
  bool multi_gt = false, multi_dh = false;  // shared pack: several nodes per pass over it
  bool tc = false;          // bfloat16 shared pack: Lambda / [Bbar; L] of delta launches on tensor cores
  bool tc_gt = false;       // ... and [Bbar; L]' y of delta launches (node-parallel schedule)
  size_t smem_gt_tc = 0;
  size_t smem_tc = 0;
  int grid_tc = 1, tn = 64;  // tensor-core launch: CTAs, nodes per GEMM
  size_t smem_mgt = 0, smem_mdh = 0;
  int grid_multi = 1;
  // hybrid schedule: the backward sweep up to r runs as the chain kernel in MODE_GT
  int grid_chain = 1, stages_chain = 0;
  size_t smem_chain = 0;
  // profiling: when set, an event is recorded before the first and after every kernel
  // of a launch_iter call (kernels_per_call + 1 events)
  cudaEvent_t* events = nullptr;
};
// kernels one launch_iter call enqueues
inline int kernels_per_call(const LaunchCfg& c, int mode) {
  if (c.schedule == SCHED_CHAIN) return 1;
  const int bwd = c.schedule == SCHED_HYBRID ? 2 : c.schedule == SCHED_FUSED ? 1 : 4;
  return 1 + ((mode & MODE_PROX) ? 1 : 0) + ((mode & MODE_BWD) ? bwd : 0);
}

// Kernel launchers (kernels.cu).  prec: smpc_precision.
// tc_width: nodes per tensor-core GEMM of a bfloat16 shared-pack factor (16, 32, 64; 0: by
// the tree size)
LaunchCfg iter_config(int prec, const IterArgs& a, int num_sms, int schedule = SCHED_CHAIN, int tc_width = 0);
int launch_iter(int prec, const IterArgs& a, const LaunchCfg& cfg, int nu, int mode, void* stream);
int launch_pack(int prec, int n, int n_k, int n_v, const double* K, const double* Lam, const double* prob,
                void* packs, long long pack_stride, void* stream);
struct CostArgs {
  int n, N, n_x, n_u, n_d, n_v;  // N: rows of stage-indexed data (sum of the trees' horizons)
  const int* parent;
  const int* stage;              // per node: its row of the stage-indexed data
  const int* tree_of;            // per node: its tree (q has one previous input per tree)
  const int* child_begin;
  const int* child_count;
  const double* prob;
  const double* pbar;
  const double* Pu;       // n_u x n_d
  const double* Pe;       // n_x x n_d
  const double* Rhat;     // n_u x n_v
  const double* L;        // n_u x n_v
  const double* alpha1;   // n_u
  double W_alpha;
  const double* dhat;     // N x n_d
  const double* eps;      // n x n_d
  const double* alpha2;   // N x n_u
  const double* q;        // n_u
  double* uhat64;         // n x n_u scratch
  double* abar;           // N x n_v scratch
  void* uhat;             // outputs in the vector type
  void* e;
  void* beta;
};
int launch_cost_update(int prec, const CostArgs& a, void* stream);
int launch_copy_final_y(int prec, const IterArgs& a, int max_iters, void* dst, void* stream);
long long pack_entries(int prec, int n_k, int n_v);
int launch_init_duals(int prec, const IterArgs& a, int warm, void* stream);
// Shards: out[j] = the sums over this GPU's chain heads below cut parent j of their s
// (n_x) and r (n_v), heads listed in CSR form (cut_off, cut_heads); and the scatter of the
// exchanged totals: for cut parent j, the first chain child in (chl_off, chl) takes the
// total, the other chain children zero, in spub / rpub.
int launch_cut_sums(int prec, const IterArgs& a, int n_cut, const int* cut_off, const int* cut_heads, void* out,
                    void* stream);
int launch_cut_scatter(int prec, const IterArgs& a, int n_cut, const int* chl_off, const int* chl, const void* in,
                       void* stream);
int launch_convert(int prec, const double* src, void* dst, long long count, void* stream);
size_t vec_size(int prec);

// Per-kernel timing of full iterations (smpc_profile_solve): kStageEvents events per
// iteration, read once the solve has finished so that launches still run ahead.
constexpr int kProfileMaxIters = 4096;  // iterations of one profiling solve (events per iteration below)
struct Profile {
  static constexpr int kStageEvents = 7;
  std::vector<cudaEvent_t> ev;  // capacity x kStageEvents
  int capacity = 0;
  int count = 0;
  int stages = 0;
};

// The launch plan of one solve (api.cpp): iteration launches nu >= polish_from of a
// SMPC_BF16 factor run the float32-pack kernel on the same vectors (args32, cfg32).
struct IterPlan {
  int prec = SMPC_FP64;
  IterArgs args{}, args32{};
  LaunchCfg cfg, cfg32;
  int polish_from = 0x7fffffff;
  int anchor_every = 0;  // > 0: anchored solve (SMPC_BF16)
  Profile* profile = nullptr;
  int kernels = 0;  // kernels enqueued through launch_planned
};
constexpr size_t kStateSize = 8;  // bytes per dual-state entry (float64, or two float32)
size_t mat_size(int prec);

}  // namespace smpc

namespace smpc {
// The parts of smpc_solve around its iteration chunks (api.cpp), shared with the batch
// solve (batch.cpp): solve_begin checks the call, plans the launches and enqueues the
// step-data upload, the cost update, the initial duals and the per-solve flags;
// solve_end enqueues the tail launch, the final dual and the outputs.
int solve_begin(smpc_factor_t* f, const smpc_step_data* data, const smpc_solve_opts* opts, cudaStream_t s,
                IterPlan* plan, IterArgs* args);
int solve_end(smpc_factor_t* f, IterPlan& plan, const IterArgs& a, int launched, smpc_result* res, cudaStream_t s);
// Validates polish_iters and the kernel configuration; SMPC_ENOTSUP when the network
// does not fit the shared-memory pipeline.
int plan_iters(const smpc_factor_t* f, const IterArgs& a, const smpc_solve_opts& opts, IterPlan* plan);
int launch_planned(IterPlan& plan, int nu, int mode, void* stream);
// Copies the final dual of the factor's last solve (vector type) to dst; synchronous.
int copy_final_y(smpc_factor_t* f, void* dst);
}  // namespace smpc

// Factor state shared by the solve entry points (api.cpp, noalloc.cu).
struct smpc_factor_t {
  const smpc_tree* tree = nullptr;
  int prec = SMPC_FP64;
  int n = 0, N = 0, n_x = 0, n_u = 0, n_d = 0, n_e = 0, n_v = 0, n_k = 0, nd = 0;
  int R = 1;  // trees of the (forest) tree; N is the number of stage-indexed data rows
  size_t vs = 8, ms = 8;
  long long pack_stride = 0;
  double lambda = 0;
  double W_alpha = 0;
  smpc::HostFactor hf;
  std::vector<void*> allocs;
  size_t device_bytes = 0;  // sum of this factor's device allocations
  // device
  void* packs = nullptr;
  bool shared_packs = false;  // one pack [Bbar; L | Lambda] for every node, scaled by pscale
  void* pscale = nullptr;     // shared packs: per node 1 / (2 p_n), vector type
  void* packs32 = nullptr;    // SMPC_BF16 only: float32 packs (anchor and polish launches)
  long long pack_stride32 = 0;
  void *ha = nullptr, *wa = nullptr;  // SMPC_BF16 only: anchor h and w, n x n_k each
  double *K64 = nullptr, *Lam64 = nullptr, *Pu = nullptr, *Pe = nullptr, *Rhat = nullptr, *L = nullptr;
  double *alpha1 = nullptr, *uhat64 = nullptr, *abar = nullptr;
  double *d_p = nullptr, *d_q = nullptr, *d_dhat = nullptr, *d_eps = nullptr, *d_alpha2 = nullptr;
  void *ybuf0 = nullptr, *ybuf1 = nullptr, *wbuf = nullptr, *h = nullptr, *uhat = nullptr, *e = nullptr, *beta = nullptr;
  void *spub = nullptr, *rpub = nullptr, *uout = nullptr, *xout = nullptr;
  void *step_s = nullptr, *step_z = nullptr, *step_p = nullptr, *mu_s = nullptr;
  void *inv_s = nullptr, *inv_z = nullptr, *inv_p = nullptr;
  std::vector<double> mu_host;
  void *x_s = nullptr, *x_min = nullptr, *x_max = nullptr, *u_min = nullptr, *u_max = nullptr, *p0 = nullptr;
  void* A = nullptr;  // dynamics matrix in the vector type, NULL for A = I (tank mass balance)
  double gamma_d = 0;
  int* counters = nullptr;
  int* flags = nullptr;
  int* flags_host = nullptr;  // pinned, 2 x 2 ints
  unsigned long long* res = nullptr;
  unsigned long long* res_tree = nullptr;  // forests: cap x R x 3 per-tree residuals
  int* tree_done = nullptr;                // forests: R per-tree iteration counts (-1 running)
  double* cvec = nullptr;
  double* theta = nullptr;    // theta_nu beside cvec (ergodic average)
  void *xbar = nullptr, *ubar = nullptr;  // ergodic averages, allocated by the first solve that asks
  int cap = 0;                // iterations the res/cvec buffers hold
  int cvec_for = -1;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaStream_t last_stream = nullptr;
  int last_launches = 0;
  int num_sms = 0;
  int schedule = smpc::SCHED_CHAIN;  // iteration schedule in use
  float tuned_ms[5] = {0, 0, 0, 0, 0};  // per schedule: ms per iteration measured when the factor chose
  int tc_width = 0;                   // bfloat16 shared packs: nodes per tensor-core GEMM (0: none)
  float tc_ms[3] = {0, 0, 0};         // ms per delta iteration measured for widths 16, 32, 64
  smpc::Profile* profile = nullptr;  // set while smpc_profile_solve runs
  bool solved_once = false;
  unsigned long long wait_ns = 2000000000ull;  // IterArgs::wait_ns (SMPC_PIPELINE_WAIT_NS)
  // the factor's last solve ran through smpc_solve_static: its residual history and stop
  // flags live in the static scratch, not in res / flags, so smpc_solve_info refuses it
  bool last_static = false;
  // captured iteration chunks (use_graph): key {first iteration, end, max_iters, tol bits,
  // polish_iters, anchor_every, ergodic} -> executable graph and its kernel count
  struct ChunkGraph {
    cudaGraphExec_t exec = nullptr;
    int kernels = 0;
  };
  std::map<std::array<long long, 7>, ChunkGraph> graphs;
  cudaStream_t capture_stream = nullptr;  // graphs are captured here, launched on the solve's stream
  bool graphs_off = false;                // a capture failed: plain launches from then on
  void drop_graphs() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second.exec);
    graphs.clear();
  }

  template <typename T>
  int alloc(T** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    void* q = nullptr;
    const cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();  // not sticky: clear it so that later launch checks do not see it
      smpc::set_error("cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? SMPC_ENOMEM : SMPC_ECUDA;
    }
    allocs.push_back(q);
    device_bytes += bytes;
    *p = static_cast<T*>(q);
    return SMPC_OK;
  }
  ~smpc_factor_t() {
    drop_graphs();
    if (capture_stream) cudaStreamDestroy(capture_stream);
    for (void* p : allocs) cudaFree(p);
    if (flags_host) cudaFreeHost(flags_host);
    for (auto& v : ev)
      if (v) cudaEventDestroy(v);
  }
};
