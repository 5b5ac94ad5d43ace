// smpc_solve_static: the solve of smpc_solve without any memory allocation.
//
// A model-predictive controller calls the solver once per sampling period and must
// return its move before the period ends (Alg. 2).  Such callers cannot allocate
// device memory inside that loop: cudaMalloc and cudaFree may synchronize the whole
// device and take unbounded time, and deployments with a fixed device-memory budget
// forbid allocation after start-up.  smpc_solve may allocate when a solve asks for
// more iterations than any earlier one; this entry point never allocates (device or
// host).  The per-iteration scratch of the iteration kernel lives in the file-scope
// array below instead of library-allocated buffers; the factor (created during the
// caller's set-up) still supplies the packs, duals, step buffers and outputs.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "smpc_internal.h"

namespace smpc {
namespace {

constexpr size_t kStaticScratchBytes = SMPC_STATIC_SCRATCH_BYTES;

// Scratch shared by every smpc_solve_static call on a device.  Every GPU that loads the
// library holds these 16 MiB until the process exits.  In host code the name is only a
// stand-in: the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_solve_scratch[kStaticScratchBytes];

struct DeviceState {
  bool ready;
  unsigned char* base;  // device address of g_solve_scratch on that device
  int theta_len;        // leading entries of the theta table valid in the array
};
constexpr int kMaxDevices = 64;
DeviceState g_dev[kMaxDevices];
std::mutex g_mutex;

// c_nu = theta_nu (1/theta_{nu-1} - 1), theta_0 = theta_{-1} = 1 (eq. optim:theta:update),
// the same recursion smpc_solve evaluates on the host.
__global__ void theta_table_kernel(double* c, int n) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double tp = 1.0, t = 1.0;
  for (int nu = 0; nu < n; ++nu) {
    c[nu] = t * (1.0 / tp - 1.0);
    const double tn = 0.5 * (sqrt(t * t * t * t + 4.0 * t * t) - t * t);
    tp = t;
    t = tn;
  }
}

size_t a256(size_t v) { return (v + 255) / 256 * 256; }

struct Layout {
  size_t cvec, res, counters, flags, wbuf, h, spub, rpub, total;
};

Layout layout(const smpc_factor_t* f, int iters) {
  Layout L;
  size_t off = 0;
  L.cvec = off;  // first, so that a longer table written by an earlier call stays in place
  off += a256(sizeof(double) * ((size_t)iters + 3));
  L.res = off;
  off += a256(sizeof(unsigned long long) * 3 * ((size_t)iters + 2));
  L.counters = off;
  off += a256(sizeof(int) * (size_t)f->n);
  L.flags = off;
  off += a256(sizeof(int) * 4);
  L.wbuf = off;
  off += a256(f->vs * (size_t)f->n * f->n_k);
  L.h = off;
  off += a256(f->vs * (size_t)f->n * f->n_k);
  L.spub = off;
  off += a256(f->vs * (size_t)f->n * f->n_x);
  L.rpub = off;
  off += a256(f->vs * (size_t)f->n * f->n_v);
  L.total = off;
  return L;
}

bool host_side(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return at.type != cudaMemoryTypeDevice;
}

bool finite_host(const double* p, size_t n) {
  if (!host_side(p)) return true;  // device-resident data is checked on the device
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

#define SCK(call)                                                                  \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      set_error("%s failed: %s", #call, cudaGetErrorString(e_));                   \
      return SMPC_ECUDA;                                                           \
    }                                                                              \
  } while (0)
#define STRY(expr)                  \
  do {                              \
    const int rc_ = (expr);         \
    if (rc_ != SMPC_OK) return rc_; \
  } while (0)

}  // namespace
}  // namespace smpc

using namespace smpc;

extern "C" int smpc_solve_static(smpc_factor_t* f, const smpc_step_data* data, const smpc_solve_opts* opts,
                                 smpc_result* res, void* stream) {
  if (!f || !data || !opts || !res) {
    set_error("NULL argument");
    return SMPC_EINVAL;
  }
  if (!data->p || !data->q || !data->alpha2 || (f->n_d > 0 && !data->dhat)) {
    set_error("step data needs p, q, dhat and alpha2");
    return SMPC_EINVAL;
  }
  if (opts->max_iters < 1 || opts->max_iters > SMPC_MAX_ITERS || !(opts->tol >= 0)) {
    set_error("max_iters must be in [1, %d] and tol >= 0", SMPC_MAX_ITERS);
    return SMPC_EINVAL;
  }
  if (opts->ergodic) {
    set_error("smpc_solve_static does not keep the ergodic average (use smpc_solve)");
    return SMPC_EINVAL;
  }
  const int n = f->n, N = f->N, n_x = f->n_x, n_u = f->n_u, n_d = f->n_d;
  const int iters = opts->max_iters;
  const Layout L = layout(f, iters);
  if (L.total > kStaticScratchBytes) {
    set_error("this solve needs %zu bytes of scratch; the static scratch of smpc_solve_static holds %zu bytes "
              "(use fewer iterations, a smaller tree, or smpc_solve)",
              L.total, kStaticScratchBytes);
    return SMPC_EINVAL;
  }
  if (!finite_host(data->p, (size_t)f->R * n_x) || !finite_host(data->q, (size_t)f->R * n_u) ||
      !finite_host(data->alpha2, (size_t)N * n_u) ||
      (n_d && !finite_host(data->dhat, (size_t)N * n_d)) || (data->eps && n_d && !finite_host(data->eps, (size_t)n * n_d))) {
    set_error("step data contains non-finite values");
    return SMPC_EINVAL;
  }
  int dev = 0;
  SCK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal %d beyond the %d devices smpc_solve_static keeps state for", dev, kMaxDevices);
    return SMPC_ENOTSUP;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // a stream under capture only records the table kernel: the table is then written
  // whenever the graph runs, so such a call always records it and leaves the recorded
  // length unknown
  cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
  SCK(cudaStreamIsCapturing(s, &capture));
  const bool capturing = capture != cudaStreamCaptureStatusNone;
  unsigned char* base = nullptr;
  bool need_theta = false;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    DeviceState& st = g_dev[dev];
    if (!st.ready) {  // once per device, with that device current
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_solve_scratch);
      if (e != cudaSuccess || p == nullptr) {
        set_error("cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
        return SMPC_ECUDA;
      }
      st.base = static_cast<unsigned char*>(p);
      st.theta_len = 0;
      st.ready = true;
    }
    base = st.base;
    need_theta = capturing || st.theta_len < iters + 3;
  }
  double* cvec = reinterpret_cast<double*>(base + L.cvec);
  unsigned long long* resv = reinterpret_cast<unsigned long long*>(base + L.res);
  int* counters = reinterpret_cast<int*>(base + L.counters);
  int* flags = reinterpret_cast<int*>(base + L.flags);

  // iteration-kernel arguments: the factor's state, the scratch from the static array.
  // The launch plan (with its option checks) comes before any device work, so that a
  // call refused for its options leaves the factor's duals as they were.
  const smpc_tree* t = f->tree;
  IterArgs a{};
  std::memset(&a, 0, sizeof a);
  a.n = n;
  a.n_x = n_x;
  a.n_u = n_u;
  a.n_v = f->n_v;
  a.n_k = f->n_k;
  a.n_chains = (int)t->chain_parent.size();
  a.n_top = (int)t->top_nodes.size();
  a.parent = t->dev.parent;
  a.child_begin = t->dev.child_begin;
  a.child_count = t->dev.child_count;
  a.chain_off = t->dev.chain_off;
  a.chain_node = t->dev.chain_node;
  a.chain_parent = t->dev.chain_parent;
  a.top_nodes = t->dev.top_nodes;
  a.top_expect = t->dev.top_expect;
  a.path_off = t->dev.path_off;
  a.path_node = t->dev.path_node;
  a.tree_of = t->dev.tree_of;
  a.seg = t->dev.seg;
  a.pscale = f->pscale;
  a.packs = f->packs;
  a.pack_stride = f->pack_stride;
  a.ybuf0 = f->ybuf0;
  a.ybuf1 = f->ybuf1;
  a.uhat = f->uhat;
  a.e = f->e;
  a.beta = f->beta;
  a.uout = f->uout;
  a.xout = f->xout;
  a.step_s = f->step_s;
  a.step_z = f->step_z;
  a.step_p = f->step_p;
  a.inv_s = f->inv_s;
  a.inv_z = f->inv_z;
  a.inv_p = f->inv_p;
  a.mu_s = f->mu_s;
  a.x_s = f->x_s;
  a.x_min = f->x_min;
  a.x_max = f->x_max;
  a.u_min = f->u_min;
  a.u_max = f->u_max;
  a.p0 = f->p0;
  a.A = f->A;
  a.gamma_d = f->gamma_d;
  a.tol = opts->tol;
  a.wbuf = base + L.wbuf;
  a.h = base + L.h;
  a.spub = base + L.spub;
  a.rpub = base + L.rpub;
  a.cvec = cvec;
  a.res = resv;
  a.counters = counters;
  a.flags = flags;
  a.wait_ns = f->wait_ns;
  // one residual for a whole forest here (no stop per tree): the per-tree record is
  // read by the warm start below, then cleared
  a.R = f->R;
  a.res_tree = nullptr;
  a.tree_done = f->tree_done;
  IterPlan plan;
  STRY(plan_iters(f, a, *opts, &plan));

  if (need_theta) {
    theta_table_kernel<<<1, 1, 0, s>>>(cvec, iters + 3);
    SCK(cudaGetLastError());
  }
  {
    // the regions behind the table move with the iteration count: only this call's table
    // length is known to survive it, and only once its table launch has been enqueued
    std::lock_guard<std::mutex> lock(g_mutex);
    g_dev[dev].theta_len = capturing ? 0 : iters + 3;
  }
  // step data -> the factor's device buffers (no allocation)
  SCK(cudaMemcpyAsync(f->d_p, data->p, sizeof(double) * f->R * n_x, cudaMemcpyDefault, s));
  SCK(cudaMemcpyAsync(f->d_q, data->q, sizeof(double) * f->R * n_u, cudaMemcpyDefault, s));
  if (n_d) SCK(cudaMemcpyAsync(f->d_dhat, data->dhat, sizeof(double) * (size_t)N * n_d, cudaMemcpyDefault, s));
  if (data->eps && n_d)
    SCK(cudaMemcpyAsync(f->d_eps, data->eps, sizeof(double) * (size_t)n * n_d, cudaMemcpyDefault, s));
  SCK(cudaMemcpyAsync(f->d_alpha2, data->alpha2, sizeof(double) * (size_t)N * n_u, cudaMemcpyDefault, s));
  STRY(launch_convert(f->prec, f->d_p, f->p0, (long long)f->R * n_x, s));
  CostArgs c;
  std::memset(&c, 0, sizeof c);
  c.n = n;
  c.N = N;
  c.n_x = n_x;
  c.n_u = n_u;
  c.n_d = n_d;
  c.n_v = f->n_v;
  c.parent = f->tree->dev.parent;
  c.stage = f->tree->dev.row;
  c.tree_of = f->tree->dev.tree_of;
  c.child_begin = f->tree->dev.child_begin;
  c.child_count = f->tree->dev.child_count;
  c.prob = f->tree->dev.prob;
  c.pbar = f->tree->dev.pbar;
  c.Pu = f->Pu;
  c.Pe = f->Pe;
  c.Rhat = f->Rhat;
  c.L = f->L;
  c.alpha1 = f->alpha1;
  c.W_alpha = f->W_alpha;
  c.dhat = f->d_dhat;
  c.eps = f->d_eps;
  c.alpha2 = f->d_alpha2;
  c.q = f->d_q;
  c.uhat64 = f->uhat64;
  c.abar = f->abar;
  c.uhat = f->uhat;
  c.e = f->e;
  c.beta = f->beta;
  STRY(launch_cost_update(f->prec, c, s));

  {
    // warm start reads the factor's own record of its last final iterate
    IterArgs ai = a;
    ai.flags = f->flags;
    STRY(launch_init_duals(f->prec, ai, (opts->warm_start && f->solved_once) ? 1 : 0, s));
  }
  SCK(cudaMemsetAsync(f->tree_done, 0xff, sizeof(int) * (size_t)f->R, s));
  // what must start at zero (the array keeps the previous call's contents)
  SCK(cudaMemsetAsync(counters, 0, sizeof(int) * (size_t)n, s));
  SCK(cudaMemsetAsync(flags, 0xff, sizeof(int), s));
  SCK(cudaMemsetAsync(flags + 1, 0, sizeof(int), s));
  SCK(cudaMemsetAsync(resv, 0, sizeof(unsigned long long) * 3 * ((size_t)iters + 2), s));
  const int chunk = opts->check_every > 0 ? opts->check_every : 128;
  int launched = 0, chunks = 0;
  bool stop = false;
  while (launched < iters && !stop) {
    const int upto = iters < launched + chunk ? iters : launched + chunk;
    for (int nu = launched; nu < upto; ++nu)
      STRY(launch_planned(plan, nu, MODE_BWD | MODE_CHECK | (nu > 0 ? MODE_PROX : 0), s));
    launched = upto;
    const int slot = chunks & 1;
    if (chunks >= 2) {
      SCK(cudaEventSynchronize(f->ev[slot]));
      if (f->flags_host[2 * slot] >= 0 || f->flags_host[2 * slot + 1] != 0) stop = true;
    }
    SCK(cudaMemcpyAsync(f->flags_host + 2 * slot, flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    SCK(cudaEventRecord(f->ev[slot], s));
    ++chunks;
  }
  STRY(launch_planned(plan, launched, MODE_PROX | MODE_CHECK, s));
  STRY(launch_copy_final_y(f->prec, a, launched, res->y, s));
  // keep the factor's record of its final iterate current (warm starts of either entry point)
  SCK(cudaMemcpyAsync(f->flags, flags, 2 * sizeof(int), cudaMemcpyDeviceToDevice, s));
  if (res->u) SCK(cudaMemcpyAsync(res->u, f->uout, (size_t)n * n_u * f->vs, cudaMemcpyDefault, s));
  if (res->x) SCK(cudaMemcpyAsync(res->x, f->xout, (size_t)n * n_x * f->vs, cudaMemcpyDefault, s));
  f->solved_once = true;
  f->last_static = true;
  f->last_stream = s;
  f->last_launches = 6 + plan.kernels + 1 + (need_theta ? 1 : 0);
  res->launches = f->last_launches;
  res->iterations = -1;
  if (!opts->sync) return SMPC_OK;
  // completion without smpc_solve_info, which may allocate host buffers
  SCK(cudaStreamSynchronize(s));
  int fl[2];
  SCK(cudaMemcpy(fl, flags, sizeof fl, cudaMemcpyDeviceToHost));
  res->iterations = fl[0];
  if (fl[0] >= 1) {
    unsigned long long r3[3];
    SCK(cudaMemcpy(r3, resv + 3 * (size_t)(fl[0] - 1), sizeof r3, cudaMemcpyDeviceToHost));
    double v[3];
    std::memcpy(v, r3, sizeof v);
    res->rho = v[0];
    res->rho_rel = v[0] / (1.0 + (v[1] > v[2] ? v[1] : v[2]));
    if (res->history_host)  // the residual history is stored as float64 bit patterns
      SCK(cudaMemcpy(res->history_host, resv, sizeof(double) * 3 * (size_t)fl[0], cudaMemcpyDeviceToHost));
  }
  if (res->u0_host) {  // the roots' inputs (nodes 0..R-1), one tree at a time
    for (int r = 0; r < f->R; ++r) {
      if (f->prec == SMPC_FP64) {
        SCK(cudaMemcpy(res->u0_host + (size_t)r * n_u, static_cast<const double*>(f->uout) + (size_t)r * n_u,
                       sizeof(double) * n_u, cudaMemcpyDeviceToHost));
      } else {
        float u0[256];  // n_u <= 256 is required by the iteration kernel
        SCK(cudaMemcpy(u0, static_cast<const float*>(f->uout) + (size_t)r * n_u, sizeof(float) * n_u,
                       cudaMemcpyDeviceToHost));
        for (int i = 0; i < n_u; ++i) res->u0_host[(size_t)r * n_u + i] = u0[i];
      }
    }
  }
  if (fl[1] != 0) {
    set_error("solve failed on the device: %s", smpc_status_string(fl[1]));
    return fl[1];
  }
  return SMPC_OK;
}
