/*
 * smpc.h - C ABI of a GB300 (sm_103a) solver for scenario-tree stochastic MPC of
 * drinking-water networks by the accelerated dual proximal gradient method
 * (Sampathirao, Sopasakis, Bemporad, Patrinos, "GPU-accelerated stochastic
 * predictive control of drinking water networks").
 *
 * Conventions shared by every call
 * --------------------------------
 * - Matrices are dense, row-major, float64, in host memory unless stated.
 * - A scenario tree (Sec. III-C) has n_nodes nodes in breadth-first order grouped
 *   by stage: parent[0] = -1 is the root (stage 0); every other node's parent has a
 *   smaller index and sits one stage up; the parents of the nodes of one stage are
 *   non-decreasing, so the children of a node are contiguous; all leaves are at the
 *   last stage N-1, where N (the horizon) is one more than the deepest stage.
 * - A forest batches R independent problems on one network into one solve: nodes
 *   0..R-1 are the roots (parent -1), and each tree's leaves are at its own last stage
 *   N_r - 1.  Per-tree step data is stacked tree after tree (smpc_step_data).
 * - Node n at stage j holds the input u_n = u_j, the demand d_n = d_j and the
 *   state x_n = x_{j+1} of its branch; its dual block is
 *   y_n = (vsigma_n, zeta_n, psi_n) of length 2 n_x + n_u (Sec. IV-A); this is the
 *   layout that reproduces the variable counts of Table 1.
 * - Device vectors use the "vector type" of a factor: float64 when the factor's
 *   precision is SMPC_FP64, float32 for SMPC_FP32 and SMPC_BF16.  The dual iterates
 *   themselves are held internally in float64, or as float32 pairs hi + lo (about
 *   48 significant bits) for the reduced precisions, so that the small dual moves of
 *   a late iteration are not rounded away.
 * - Every call returns an smpc_status; none throws.  On failure the message of
 *   the calling thread's last error is available from smpc_last_error().
 * - Objects are owned by the library and released by the matching *_destroy.
 *   Device memory is allocated by the library with cudaMalloc on the device that
 *   is current when the object is created; all later calls on the object must be
 *   made with that device current.
 */
#ifndef SMPC_H
#define SMPC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum smpc_status {
  SMPC_OK = 0,
  SMPC_EINVAL = 1,    /* bad argument: sizes, tree shape, probabilities, NaN, ... */
  SMPC_ENOMEM = 2,    /* host or device allocation failed */
  SMPC_ECUDA = 3,     /* a CUDA runtime call failed (includes "no device") */
  SMPC_EBUSY = 4,     /* server: the request can never fit the memory budget or slots */
  SMPC_ETIMEOUT = 5,  /* a bounded device wait gave up; results are not valid */
  SMPC_EDIVERGED = 6, /* non-finite values in the iterates (e.g. infeasible coupling) */
  SMPC_ENOTSUP = 7    /* valid request outside what this build implements (e.g. A != I on schedule 4) */
} smpc_status;

typedef enum smpc_precision {
  SMPC_FP64 = 0, /* per-node matrices and vectors in float64 */
  SMPC_FP32 = 1, /* per-node matrices and vectors in float32, float32 accumulation */
  SMPC_BF16 = 2  /* per-node matrices in bfloat16, vectors and accumulation float32 */
} smpc_precision;

typedef struct smpc_tree smpc_tree;
typedef struct smpc_factor_t smpc_factor_t;
typedef struct smpc_server smpc_server;
typedef struct smpc_batch smpc_batch;
typedef struct smpc_shard smpc_shard;

/* Flow-based network model x+ = A x + B u + G_d d, 0 = E u + E_d d (Sec. II-A,
 * eqs. model and demand-control).  A may be NULL for the identity (tank mass
 * balance), the paper's network, which every iteration schedule handles.  A general
 * A (App. B: s_n = xi_n + A' sum of the children's s, x_n = A x_parent + Bbar v_n +
 * e_n) runs on the node-parallel schedule (2) only, with one n_x x n_x mat-vec per node
 * in the s-scan and in the forward sweep.  E and Ed may be NULL when n_e = 0.  E must
 * have full row rank. */
typedef struct smpc_network {
  int32_t n_x, n_u, n_d, n_e;
  const double* A;  /* n_x * n_x or NULL (identity) */
  const double* B;  /* n_x * n_u */
  const double* Gd; /* n_x * n_d */
  const double* E;  /* n_e * n_u */
  const double* Ed; /* n_e * n_d */
} smpc_network;

/* Costs and bounds (Sec. III-A, eqs. cost:linear, cost:smooth, cost:non-smooth;
 * soft state box of eq. cost:distance; input box of eq. Sc-MPC).
 * The safety penalty of node n is mu_S,n dist(x_n | {x >= x_s}) with
 * mu_S,n = p_n W_x (l^S sits inside the expectation of eq. Sc-MPC) unless
 * safety_unweighted = 1, which uses mu_S,n = W_x as printed in eq. gzeta. */
typedef struct smpc_cost {
  double W_alpha;         /* economic scaling W_alpha */
  const double* alpha1;   /* n_u production cost alpha_1 */
  const double* W_u;      /* n_u * n_u symmetric positive definite smoothing weight */
  double W_x;             /* safety weight */
  double gamma_d;         /* soft state-box weight */
  const double* x_min;    /* n_x */
  const double* x_max;    /* n_x */
  const double* x_s;      /* n_x safety level */
  const double* u_min;    /* n_u */
  const double* u_max;    /* n_u */
  int32_t safety_unweighted;
} smpc_cost;

typedef struct smpc_factor_opts {
  int32_t precision;      /* smpc_precision of the per-node matrix packs */
  int32_t precondition;   /* 1: Jacobi diagonal scaling of the dual (Sec. IV-D); 0: none */
  double lambda;          /* > 0: use this step; 0: estimate 1/L by power iteration */
  int32_t power_iters;    /* power iterations for the estimate (0: default 200) */
  double lambda_margin;   /* estimate is divided by (1 + margin) (0: default 0.02) */
  /* Explicit per-entry steps (all three or none; host float64).  When given they
   * replace lambda and the preconditioner: step_s[n], step_z[n] are the steps of
   * node n's two distance blocks, step_p[n*n_u + i] of its input entries. */
  const double* step_s;
  const double* step_z;
  const double* step_p;
  /* 1: one pack for all nodes - [Bbar; L] and Lambda are the same at every node, only the
   * scale 1 / (2 p_n) differs and is applied to Lambda r - held in shared memory while the
   * mat-vecs run, so that the matrices leave HBM traffic; 0: one pack per node (the
   * node-indexed matrices of Alg. 1 and App. B).  Results agree to rounding. */
  int32_t shared_packs;
  /* Iteration schedule: 1 = one launch per iteration with one CTA per chain (maximal
   * leaf path) of the tree; 2 = the backward sweep as subtree scans around per-node
   * mat-vec launches, one task per node; 3 = node-parallel forward sweep and prox, a chain
   * pass up to r, and the node-parallel Lambda / [Bbar; L] launch; 4 = node-parallel forward
   * sweep and prox, then the whole backward sweep as one chain pass (every pack read once
   * per iteration); 0 = time all of them on this GPU when the factor is built and keep the
   * fastest.  Results agree to rounding. */
  int32_t schedule;
  /* SMPC_BF16 with shared_packs = 1: the Lambda and [Bbar; L] products of the delta
   * iterations (and, on the node-parallel schedule 2, their [Bbar; L]' products) run on the
   * tensor cores as GEMMs over tc_width nodes at a time (16, 32 or 64), with the vectors
   * rounded to bfloat16; 0 = time the three widths on this GPU when the factor is built and
   * keep the fastest.  Ignored otherwise.  Results are the same for every width. */
  int32_t tc_width;
} smpc_factor_opts;

/* Per-solve data (Alg. 2, steps 1-2).  float64; each pointer may address host or
 * device memory (unified addressing decides the copy direction). */
typedef struct smpc_step_data {
  const double* p;      /* R * n_x measured state x_0 of each tree */
  const double* q;      /* R * n_u previous input u_{-1} of each tree */
  const double* dhat;   /* (N_0 + ... + N_{R-1}) * n_d nominal forecast (eq. demand:tree):
                           row N_0 + ... + N_{r-1} + j is stage j of tree r */
  const double* eps;    /* n_nodes * n_d forecast errors of the nodes, or NULL to
                           keep those uploaded by the previous solve (zero at first) */
  const double* alpha2; /* (N_0 + ... + N_{R-1}) * n_u time-varying price, rows as dhat */
} smpc_step_data;

/* Largest iteration cap a solve accepts: the per-iteration tables a solve keeps (the
 * extrapolation coefficients on the host and the device, the residual history) grow with
 * it, and larger caps are refused with SMPC_EINVAL before anything is allocated. */
#define SMPC_MAX_ITERS (1 << 26)

typedef struct smpc_solve_opts {
  int32_t max_iters;    /* iteration cap, 1 .. SMPC_MAX_ITERS */
  double tol;           /* stop at the first iterate with rho_rel <= tol (0: run max_iters) */
  int32_t warm_start;   /* 1: start from the duals the previous solve left on the device */
  int32_t check_every;  /* host polls the stop flag every this many iterations (0: 128) */
  int32_t sync;         /* 1: wait for the stream, fill the host outputs, check errors */
  /* SMPC_BF16 factors only (other precisions ignore both).  The solve step is affine
   * in w, h(w) = h(w_a) + h_lin(w - w_a): every anchor_every-th iteration (0: 16) is
   * an anchor that evaluates the whole step at w_a = w^nu with the factor's float32
   * packs, and the iterations between apply the bfloat16 packs to w - w_a only.  The
   * iteration's fixed points are those of the float32 packs, while bfloat16 carries
   * the matrix traffic of all other iterations.  The last polish_iters iterations
   * (0 <= polish_iters <= max_iters) are all anchors: the final set of iterations
   * with float32 matrices. */
  int32_t polish_iters;
  int32_t anchor_every;
  /* 1: enqueue each chunk of check_every iterations as a CUDA graph, captured the
   * first time the factor runs that chunk with these max_iters, tol, polish_iters and
   * anchor_every, and replayed by later solves of the factor with the same settings
   * (the closed loop of Alg. 2 solves every step with the same ones).  A graph that
   * cannot be captured turns graphs off for the factor (plain launches, same results).
   * Each graph is kept until the factor is destroyed (or its iteration buffers grow), so
   * solves with many different settings accumulate graphs: one per chunk and setting.
   * 0: plain launches.  smpc_solve only; smpc_solve_static ignores it. */
  int32_t use_graph;
  /* 1: also keep the ergodic primal average of Sec. IV-A (after eq. apg-iteration),
   * zbar^nu = (1 - theta_nu) zbar^{nu-1} + theta_nu z^nu with zbar^0 = z^0, over the
   * iterates of this solve (theta restarts at every solve, warm or cold), in the vector
   * type; a forest's tree stops averaging at its own stop.  Costs one read and write of
   * zbar per node and iteration in the prox launch; the first such solve on a factor
   * allocates its n_nodes * (n_x + n_u) entries.  Returned through smpc_result's xbar and
   * ubar.  0: not kept.  smpc_solve_static refuses it (SMPC_EINVAL). */
  int32_t ergodic;
} smpc_solve_opts;

/* Outputs.  Device pointers may be NULL (not copied).  Host outputs are filled
 * only when opts->sync = 1. */
typedef struct smpc_result {
  void* u;              /* device, n_nodes * n_u of the vector type: last z^nu inputs */
  void* x;              /* device, n_nodes * n_x: last z^nu states */
  void* y;              /* device, n_nodes * (2 n_x + n_u): final dual y^{nu+1} */
  double* u0_host;      /* host, R * n_u: each root's input u_0 (the move applied, Alg. 2 step 4) */
  double* history_host; /* host, max_iters * 3: per iteration (rho, ||Hz||_inf, ||t||_inf) */
  int32_t iterations;   /* out: iterations run */
  double rho;           /* out: ||H z - t||_inf of the last iterate (Sec. IV-E), over all trees */
  double rho_rel;       /* out: rho / (1 + max(||H z||_inf, ||t||_inf)) */
  int32_t launches;     /* out: kernel launches the solve enqueued (set on return) */
  double queue_ms;      /* out (smpc_poll only): submit to admission, host wall clock */
  double run_ms;        /* out (smpc_poll only): admission to completion, host wall clock */
  void* ubar;           /* device, n_nodes * n_u: ergodic average of u (opts->ergodic = 1 only) */
  void* xbar;           /* device, n_nodes * n_x: ergodic average of x (opts->ergodic = 1 only) */
} smpc_result;

typedef struct smpc_tree_info {
  int32_t n_nodes, horizon, n_leaves, n_chains, n_top, max_chain_len;
  int32_t n_trees;  /* trees of a forest (1 for a single scenario tree) */
} smpc_tree_info;

/* Validate a scenario tree (Sec. III-C) and upload it.  prob[n] is p_n, the
 * probability of reaching node n; children's probabilities must add up to the
 * parent's (relative 1e-12) and the root's must be 1.  prob = NULL means
 * equiprobable scenarios.  Inputs are copied.
 * Errors: SMPC_EINVAL (shape, order, probabilities), SMPC_ECUDA, SMPC_ENOMEM. */
int smpc_tree_create(int32_t n_nodes, const int32_t* parent, const double* prob, smpc_tree** out);
int smpc_tree_info_get(const smpc_tree* tree, smpc_tree_info* info);
void smpc_tree_destroy(smpc_tree* tree);

/* Offline factor step (App. A and App. B; Alg. 2 lines 1-2), in float64 on the
 * host: L = orthonormal basis of null(E), B_bar = B L, R_hat = W_u L,
 * R_bar = L' R_hat, Cholesky of R_bar, Lambda = -R_bar^{-1}; then per-node packs
 * [B_bar; L] (n_x + n_u) x n_v and Lambda / (2 p_n) (n_v x n_v, Alg. 1's
 * node-indexed factor matrices) in the requested precision on the device, the
 * Jacobi scaling (Sec. IV-D) and the step lambda = 1/L_{H_D} (power iteration
 * on the device, unless given).  An SMPC_BF16 factor also keeps float32 packs for
 * the anchor and polish iterations of smpc_solve_opts.  The tree must outlive the factor.
 * Errors: SMPC_EINVAL (sizes, NaN, E rank deficient, W_u not SPD),
 *         SMPC_ENOTSUP (A != I with a schedule other than 0 or 2), SMPC_ENOMEM, SMPC_ECUDA. */
int smpc_factor(const smpc_tree* tree, const smpc_network* net, const smpc_cost* cost,
                const smpc_factor_opts* opts, smpc_factor_t** out);
void smpc_factor_destroy(smpc_factor_t* fac);
/* The steps in use: lambda (the scalar of Sec. IV-D; 0 when explicit steps were
 * given) and, when the pointers are not NULL, the per-entry steps (host float64,
 * shapes as in smpc_factor_opts). */
int smpc_factor_steps(const smpc_factor_t* fac, double* lambda, double* step_s, double* step_z,
                      double* step_p);
/* Returns the schedule the factor uses (1 to 4, see smpc_factor_opts.schedule), or minus
 * SMPC_EINVAL for a NULL factor.  When ms_per_iter is not NULL, ms_per_iter[0..3] receive the
 * measured ms per iteration of schedules 1, 2, 3 and 4 when the factor chose among them (0
 * when it did not time them). */
int smpc_factor_schedule(const smpc_factor_t* fac, double* ms_per_iter);

/* One SMPC solve (Alg. 2 step 3): the cost update of App. A on the device from
 * the step data, then APG iterations (eq. apg-iteration) with Algorithm 1 as the
 * solve step and the prox of App. C, until rho_rel <= tol or max_iters.
 * Stream-ordered on `stream` (a cudaStream_t; NULL = legacy default stream).
 * Calls on the same factor must not overlap.
 * Errors: SMPC_EINVAL, SMPC_ECUDA, SMPC_ETIMEOUT, SMPC_EDIVERGED (sync only). */
int smpc_solve(smpc_factor_t* fac, const smpc_step_data* data, const smpc_solve_opts* opts,
               smpc_result* res, void* stream);

/* smpc_solve without memory allocation.  The paper has no counterpart: it exists for
 * callers that cannot allocate device memory while they run.  A model-predictive
 * controller solves once per sampling period and must return its move within the
 * period (Alg. 2); cudaMalloc and cudaFree may synchronize the whole device and take
 * unbounded time, and deployments with a fixed device-memory budget forbid allocation
 * after start-up.  smpc_solve may allocate when a solve asks for more iterations than
 * any earlier solve on its factor; smpc_solve_static allocates nothing, on the device
 * or the host.  The factor, created during the caller's set-up, still supplies the
 * packs, duals and step buffers, and the caller passes inputs and outputs as for
 * smpc_solve (same arguments, results and errors).
 *
 * The iteration kernel's scratch (theta table, residual history, arrival counters, stop
 * and error flags, w, h and the published s and r of the tree reduction) lives in one
 * static device array of SMPC_STATIC_SCRATCH_BYTES (16 MiB) that every GPU which loads
 * the library holds until the process exits.  A solve needing more - about
 * 32 (max_iters + 3) + 4 n_nodes + vs n_nodes (3 n_x + 2 n_u + n_v) bytes, vs = 8 for
 * SMPC_FP64 and 4 otherwise - is refused with SMPC_EINVAL before any device work.
 * The first call on a device resolves the array's device address (cudaGetSymbolAddress)
 * and should come before any stream capture.  All calls, on any factor and any stream,
 * share the array and leave their contents in it; each call clears what must start at
 * zero.  Calls that overlap on the GPU race on the array: the caller must serialize
 * them.  warm_start continues from the last solve of the same factor by either entry point.
 * Host outputs (iterations, rho, u0_host, history_host) are filled with opts->sync = 1;
 * smpc_solve_info completes smpc_solve only. */
#define SMPC_STATIC_SCRATCH_BYTES (16u << 20)
int smpc_solve_static(smpc_factor_t* fac, const smpc_step_data* data, const smpc_solve_opts* opts,
                      smpc_result* res, void* stream);

/* Batched solves (Sec. IV-B's stage parallelism carried across independent problems):
 * smpc_batch_create groups `count` factors - single trees or forests (several trees on one
 * network, see smpc_tree_create), on any mix of networks and precisions - that are then
 * solved together.  smpc_batch_solve runs the solve of smpc_solve for every factor k with
 * its own step data data[k] and the shared opts, and writes res[k]: each chunk of
 * opts->check_every iterations is one launch for the whole batch - with
 * opts->use_graph = 1 a CUDA graph whose parallel branches are the factors' kernels for
 * those iterations, captured the first time the batch runs that chunk with these settings
 * and replayed by later solves; with use_graph = 0 the same kernels on one stream per
 * factor between a fork and a join on `stream`.  Every factor keeps its own state and
 * stop: a factor (or a forest's tree) whose residual met tol keeps its iterates and its
 * kernels return at once; the batch ends when every factor has stopped or at max_iters.
 * Results per factor, exactly as smpc_solve on that factor alone (including
 * smpc_solve_trees for forests).  The factors must outlive the batch and a factor may
 * appear in one batch solve at a time; calls on the same batch must not overlap.
 * Errors: as smpc_solve (the first failing factor's), SMPC_EINVAL for a NULL or
 * repeated factor, SMPC_ECUDA, SMPC_ENOMEM. */
int smpc_batch_create(int32_t count, smpc_factor_t* const* factors, smpc_batch** out);
int smpc_batch_solve(smpc_batch* batch, const smpc_step_data* data, const smpc_solve_opts* opts, smpc_result* res,
                     void* stream);
void smpc_batch_destroy(smpc_batch* batch);

/* Shards: one scenario tree split over several GPUs, one process per GPU (Sec. IV-B: the
 * nodes of a stage are independent given their children's sums).  Every GPU creates the
 * tree and factor of the whole problem, then a shard that owns the chains (maximal leaf
 * paths, numbered as smpc_tree_info's n_chains) [chain_begin, chain_end); the top nodes
 * above the chains are replicated on every GPU.  A sharded solve is driven by the caller,
 * who owns the exchange between the GPUs:
 *   smpc_shard_begin(shard, data, opts, residuals, stream)   - smpc_solve's set-up;
 *   for nu = 0, 1, ...:
 *     smpc_shard_step(shard, nu, 0, exchange)   - forward sweep and prox of the shard's nodes
 *         (iteration nu - 1), backward sweep along its chains (iteration nu), and into
 *         exchange (device, n_cut x (n_x + n_v) of the vector type) the sums of s and r
 *         over its chain heads below each cut parent (a top node with chain children);
 *     caller: exchange = its sum over the GPUs (allreduce, sum);
 *     smpc_shard_step(shard, nu, 1, exchange)   - the backward sweep of the top nodes with
 *         the totals, the same on every GPU;
 *     caller (nu >= 1): residuals[3 (nu - 1) .. 3 (nu - 1) + 2] = its maximum over the GPUs
 *         (allreduce, max; float64 bit patterns, so an integer maximum is the same);
 *     every so often smpc_shard_flags: once done >= 0 the solve has stopped on every GPU;
 *   smpc_shard_step(shard, n, 2, NULL) with n = the loop count - the last prox; the caller's
 *       residual maximum for iteration n - 1; then smpc_shard_finish(shard, n, res).
 * residuals: device, 3 (max_iters + 2) unsigned 64-bit, owned by the caller.  Each GPU's
 * outputs hold its own chains' and the top nodes' entries (others are not updated).  Stops
 * are the same on every GPU since every GPU reads the same residuals.  float64 and float32
 * factors of a single tree whose root is a top node; all calls on the stream of begin.
 * Errors: SMPC_EINVAL, SMPC_ENOTSUP (bfloat16, a chain starting at a root), SMPC_ENOMEM,
 * SMPC_ECUDA, and the solve's own errors from smpc_shard_finish. */
int smpc_shard_create(smpc_factor_t* fac, int32_t chain_begin, int32_t chain_end, smpc_shard** out);
int smpc_shard_info(const smpc_shard* shard, int32_t* n_cut, int32_t* width, int32_t* n_nodes);
/* The n_nodes (smpc_shard_info) nodes whose rows this shard's outputs hold, ascending:
 * the top nodes and the nodes of its own chains. */
int smpc_shard_nodes(const smpc_shard* shard, int32_t* nodes);
int smpc_shard_begin(smpc_shard* shard, const smpc_step_data* data, const smpc_solve_opts* opts,
                     unsigned long long* residuals, void* stream);
int smpc_shard_step(smpc_shard* shard, int32_t nu, int32_t phase, void* exchange);
int smpc_shard_flags(const smpc_shard* shard, int32_t* done, int32_t* error);
int smpc_shard_finish(smpc_shard* shard, int32_t launched, smpc_result* res);
void smpc_shard_destroy(smpc_shard* shard);

/* Diagnostics; the paper has no counterpart.  Runs one cold-start solve of `iters`
 * iterations (2 .. 4096; tol 0, legacy default stream) with a CUDA event between consecutive kernels
 * of every full iteration, and writes the mean device time in ms
 * of each kernel of an iteration to stage_ms[0 .. min(n, max_stages)).  n = 1 for schedule 1
 * (apg_iter), 6 for schedule 2 (forward sweep, prox and dual update, subtree scan of s,
 * [Bbar; L]' mat-vec, subtree scan of r, Lambda and [Bbar; L] mat-vecs) and 4 for schedule 3
 * (forward sweep; prox and dual update; s, [Bbar; L]' mat-vecs and r along the chains; Lambda
 * and [Bbar; L] mat-vecs) and 3 for schedule 4 (forward sweep; prox and dual update; the
 * whole backward sweep along the chains).  SMPC_BF16 anchor iterations are not timed.  Leaves
 * the factor's duals as that solve ends.  Returns n, or minus an smpc_status. */
int smpc_profile_solve(smpc_factor_t* fac, const smpc_step_data* data, int32_t iters, double* stage_ms,
                       int32_t max_stages);

/* Diagnostics; the paper has no counterpart.  Measures the fused multiply-add
 * throughput of the current GPU in TFLOP/s (2 flops per FMA) for precision SMPC_FP64
 * or SMPC_FP32: 8 CTAs of 256 threads per SM, 8 independent FMA chains per thread,
 * one launch timed with CUDA events after a warm-up launch.  This is the ceiling of a
 * solve bound by arithmetic rather than memory (float64 packs apply 2 flops per matrix
 * entry read).  Allocates and frees a small device buffer.
 * Errors: SMPC_EINVAL (other precision, NULL result), SMPC_ENOMEM, SMPC_ECUDA. */
int smpc_fma_peak(int32_t precision, double* tflops);

/* The tensor-core GEMM width (nodes per GEMM) a bfloat16 shared-pack factor uses, or 0
 * when its launches do not use the tensor cores; minus SMPC_EINVAL for a NULL factor.  When
 * ms_per_width is not NULL, ms_per_width[0..2] receive the measured ms per delta iteration
 * with widths 16, 32 and 64 (0 when not timed). */
int smpc_factor_tc_width(const smpc_factor_t* fac, double* ms_per_width);

/* Per-tree results of the factor's last smpc_solve (waits for its stream).  In a forest
 * (smpc_tree_create with R roots) every tree stops at its own first iterate whose
 * relative residual rho_rel = rho / (1 + max(||H z||_inf, ||t||_inf)) (Sec. IV-E), taken
 * over that tree's nodes alone, is <= tol: from then on the tree's iterates, outputs and
 * final dual stay as they were at that iterate while the other trees go on, and the solve
 * ends when every tree has stopped (or at max_iters).  iterations[r] receives the
 * iterations tree r ran, rho_rel[r] its relative residual at its last iterate (R entries
 * each; either pointer may be NULL).  A single tree reports the solve's own figures.
 * smpc_solve_static keeps one residual for the whole forest and no per-tree record.
 * Errors: SMPC_EINVAL (no smpc_solve yet, or the last solve was static), SMPC_ECUDA. */
int smpc_solve_trees(smpc_factor_t* fac, int32_t* iterations, double* rho_rel);

/* Completes an asynchronous solve (opts->sync = 0): waits for the stream of the
 * factor's last solve and fills the host outputs of `res` (iterations, rho,
 * rho_rel, u0_host, history_host) exactly as a synchronous solve would.
 * Errors: SMPC_EINVAL (no solve yet), SMPC_ECUDA, SMPC_ETIMEOUT, SMPC_EDIVERGED. */
int smpc_solve_info(smpc_factor_t* fac, smpc_result* res);

/* The device memory a factor holds (bytes): its packs, vectors and buffers.  This is
 * the footprint a server admits requests by. */
size_t smpc_factor_device_bytes(const smpc_factor_t* fac);

/* Serving (the paper's closed loop, Alg. 2, run for many controllers at once).  A
 * server owns max_slots execution slots, each a host worker thread with its own
 * non-blocking CUDA stream on the device current at creation.  smpc_submit queues one
 * solve of a factor and returns at once with a ticket; a queued request is admitted
 * into a free slot, in arrival order among the requests that can run, when the device
 * memory of the factors being solved plus its own factor's fits hbm_budget (bytes).
 * Admitted solves run concurrently, their kernels overlapping on the GPU, while new
 * requests keep arriving.  A factor is held from admission until smpc_poll returns its
 * ticket as done, so later requests of the same factor wait (a controller's next step
 * warm-starts, with opts->warm_start, from the duals of its previous one).  Step data
 * (host or device memory) is copied at submission; opts->sync is ignored.
 * Errors: smpc_server_create: SMPC_EINVAL, SMPC_ENOMEM, SMPC_ECUDA.
 *         smpc_submit: SMPC_EINVAL; SMPC_EBUSY when the factor alone exceeds the budget. */
int smpc_server_create(size_t hbm_budget, int32_t max_slots, smpc_server** out);
int smpc_submit(smpc_server* server, smpc_factor_t* fac, const smpc_step_data* data, const smpc_solve_opts* opts,
                uint64_t* ticket);
/* Non-blocking.  *done = 0 while the ticket is queued or running.  Once done, fills the
 * host outputs of res (iterations, rho, rho_rel, launches, queue_ms, run_ms, and u0_host /
 * history_host when not NULL) and copies u, x, y to the device pointers of res that are
 * not NULL, releases the ticket and the factor, and returns the solve's status.  res may
 * be NULL.  Errors: SMPC_EINVAL (unknown ticket), the solve's own error, SMPC_ECUDA. */
int smpc_poll(smpc_server* server, uint64_t ticket, smpc_result* res, int32_t* done);
/* Waits for the admitted solves, drops the queued ones and releases the server. */
void smpc_server_destroy(smpc_server* server);

const char* smpc_status_string(int status);
const char* smpc_last_error(void);
int smpc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SMPC_H */
