// C ABI of the SMPC solver: tree validation and decomposition, the factor step,
// preconditioning and step size (Sec. IV-D), and the solve loop (Alg. 2 step 3).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "smpc_internal.h"

namespace smpc {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

}  // namespace smpc

using namespace smpc;

#define CK(call)                                                                \
  do {                                                                          \
    cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess) {                                                    \
      set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return e_ == cudaErrorMemoryAllocation ? SMPC_ENOMEM : SMPC_ECUDA;        \
    }                                                                           \
  } while (0)

#define TRY(expr)             \
  do {                        \
    int rc_ = (expr);         \
    if (rc_ != SMPC_OK) return rc_; \
  } while (0)

namespace {

template <typename T>
int dev_upload(T** dst, const T* src, size_t count) {
  *dst = nullptr;
  if (count == 0) return SMPC_OK;
  CK(cudaMalloc(reinterpret_cast<void**>(dst), count * sizeof(T)));
  CK(cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice));
  return SMPC_OK;
}

bool finite_array(const double* p, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

// True when the host may dereference p (pageable, pinned or managed memory).
bool host_readable(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return at.type != cudaMemoryTypeDevice;
}

// Finiteness of step data that lives in host memory; device-resident data is
// checked on the device instead (non-finite iterates raise SMPC_EDIVERGED).
bool finite_if_host(const double* p, size_t n) { return !host_readable(p) || finite_array(p, n); }

void free_tree_dev(smpc::DevTree& d) {
  void* ptrs[] = {d.parent, d.stage, d.child_begin, d.child_count, d.chain_off, d.chain_node, d.chain_parent,
                  d.top_nodes, d.top_expect, d.path_off, d.path_node, d.tree_of, d.row, d.seg, d.prob, d.pbar};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  d = smpc::DevTree();
}

// Host-side validation and decomposition of a tree (no CUDA calls).
int build_tree(int32_t n, const int32_t* parent, const double* prob, smpc_tree& t) {
  if (n < 1 || !parent) {
    set_error("tree needs n_nodes >= 1 and a parent array");
    return SMPC_EINVAL;
  }
  if (parent[0] != -1) {
    set_error("parent[0] must be -1 (the root)");
    return SMPC_EINVAL;
  }
  t.n = n;
  t.parent.assign(parent, parent + n);
  t.stage.assign(n, 0);
  // a forest: the first R nodes are roots (parent -1), one per tree
  t.R = 1;
  while (t.R < n && parent[t.R] == -1) ++t.R;
  for (int m = t.R; m < n; ++m) {
    const int p = parent[m];
    if (p < 0 || p >= m) {
      set_error("parent[%d] = %d: parents must precede their children", m, p);
      return SMPC_EINVAL;
    }
    t.stage[m] = t.stage[p] + 1;
    if (t.stage[m] < t.stage[m - 1]) {
      set_error("node %d: nodes must be grouped by stage (breadth-first order)", m);
      return SMPC_EINVAL;
    }
    if (t.stage[m] == t.stage[m - 1] && m > t.R && p < parent[m - 1]) {
      set_error("node %d: parents of one stage must be non-decreasing", m);
      return SMPC_EINVAL;
    }
  }
  t.N = t.stage[n - 1] + 1;
  t.child_begin.assign(n, 0);
  t.child_count.assign(n, 0);
  for (int m = n - 1; m >= t.R; --m) {
    t.child_begin[parent[m]] = m;
    t.child_count[parent[m]]++;
  }
  // tree of every node, each tree's horizon (its deepest stage + 1) and data rows:
  // tree r's stage j reads row row_off[r] + j of the stage-indexed step data
  t.tree_of.assign(n, 0);
  std::vector<int> depth(t.R, 0);
  for (int m = 0; m < n; ++m) {
    t.tree_of[m] = m < t.R ? m : t.tree_of[parent[m]];
    depth[t.tree_of[m]] = std::max(depth[t.tree_of[m]], t.stage[m] + 1);
  }
  t.row_off.assign(t.R + 1, 0);
  for (int r = 0; r < t.R; ++r) t.row_off[r + 1] = t.row_off[r] + depth[r];
  t.rows = t.row_off[t.R];
  t.row.assign(n, 0);
  for (int m = 0; m < n; ++m) t.row[m] = t.row_off[t.tree_of[m]] + t.stage[m];
  t.n_leaves = 0;
  for (int m = 0; m < n; ++m)
    if (t.child_count[m] == 0) {
      ++t.n_leaves;
      const int last = depth[t.tree_of[m]] - 1;
      if (t.stage[m] != last) {
        set_error("leaf %d is at stage %d; all leaves of its tree must be at its last stage %d", m, t.stage[m], last);
        return SMPC_EINVAL;
      }
    }
  // probabilities
  t.prob.assign(n, 0.0);
  if (!prob) {
    std::vector<double> leaves(n, 0.0);
    for (int m = n - 1; m >= 0; --m) {
      if (t.child_count[m] == 0) leaves[m] = 1.0;
      if (m >= t.R) leaves[parent[m]] += leaves[m];
    }
    for (int m = 0; m < n; ++m) t.prob[m] = leaves[m] / leaves[t.tree_of[m]];
  } else {
    for (int m = 0; m < n; ++m) {
      if (!(std::isfinite(prob[m]) && prob[m] > 0)) {
        set_error("prob[%d] = %g must be positive and finite", m, prob[m]);
        return SMPC_EINVAL;
      }
      t.prob[m] = prob[m];
    }
    for (int r = 0; r < t.R; ++r)
      if (std::fabs(prob[r] - 1.0) > 1e-12) {
        set_error("root probability %.17g != 1 (root %d)", prob[r], r);
        return SMPC_EINVAL;
      }
    std::vector<double> csum(n, 0.0);
    for (int m = t.R; m < n; ++m) csum[parent[m]] += prob[m];
    for (int m = 0; m < n; ++m)
      if (t.child_count[m] > 0 && std::fabs(csum[m] - prob[m]) > 1e-12 * prob[m]) {
        set_error("children of node %d have probability %.17g != %.17g", m, csum[m], prob[m]);
        return SMPC_EINVAL;
      }
  }
  t.pbar = t.prob;
  for (int m = t.R; m < n; ++m) t.pbar[parent[m]] += t.prob[m];
  // chains (subtrees that are paths) and top nodes
  std::vector<char> path_sub(n, 0);
  for (int m = n - 1; m >= 0; --m)
    path_sub[m] = t.child_count[m] == 0 || (t.child_count[m] == 1 && path_sub[t.child_begin[m]]);
  t.is_top.assign(n, 0);
  std::vector<std::vector<int>> chains;
  for (int m = 0; m < n; ++m) {
    t.is_top[m] = !path_sub[m];
    if (path_sub[m] && (parent[m] < 0 || !path_sub[parent[m]])) {
      std::vector<int> c;
      for (int k = m;; k = t.child_begin[k]) {
        c.push_back(k);
        if (t.child_count[k] == 0) break;
      }
      chains.push_back(c);
    }
  }
  std::stable_sort(chains.begin(), chains.end(),
                   [](const std::vector<int>& a, const std::vector<int>& b) { return a.size() > b.size(); });
  t.chain_off.assign(1, 0);
  t.chain_node.clear();
  t.chain_parent.clear();
  t.max_chain_len = 0;
  for (auto& c : chains) {
    t.chain_node.insert(t.chain_node.end(), c.begin(), c.end());
    t.chain_off.push_back((int)t.chain_node.size());
    t.chain_parent.push_back(parent[c[0]]);
    t.max_chain_len = std::max(t.max_chain_len, (int)c.size());
  }
  t.top_nodes.clear();
  t.top_expect.assign(n, 0);
  t.path_off.assign(n + 1, 0);
  t.path_node.clear();
  for (int m = 0; m < n; ++m) {
    t.path_off[m] = (int)t.path_node.size();
    if (t.is_top[m]) {
      t.top_nodes.push_back(m);
      t.top_expect[m] = t.child_count[m] + 1;
      std::vector<int> p;
      for (int k = m; k >= 0; k = parent[k]) p.push_back(k);
      t.path_node.insert(t.path_node.end(), p.rbegin(), p.rend());
    }
  }
  t.path_off[n] = (int)t.path_node.size();
  const int n_seg = (int)(t.top_nodes.size() + t.chain_parent.size());
  t.seg.assign((size_t)n_seg * smpc::kSegInts, 0);
  for (int b = 0; b < n_seg; ++b) {
    int* d = t.seg.data() + (size_t)b * smpc::kSegInts;
    const bool top = b < (int)t.top_nodes.size();
    const int c = b - (int)t.top_nodes.size();
    const int par = top ? t.top_nodes[b] : t.chain_parent[c];
    d[0] = par;
    d[1] = par >= 0 ? t.path_off[par] : 0;
    d[2] = par >= 0 ? t.path_off[par + 1] - t.path_off[par] : 0;
    d[3] = top ? t.tree_of[par] : t.tree_of[t.chain_node[t.chain_off[c]]];
    d[4] = top ? 0 : t.chain_off[c];
    d[5] = top ? 0 : t.chain_off[c + 1] - t.chain_off[c];
  }
  return SMPC_OK;
}

int upload_tree(smpc_tree& t) {
  CK(cudaGetDevice(&t.device));
  auto& d = t.dev;
  TRY(dev_upload(&d.parent, t.parent.data(), t.n));
  TRY(dev_upload(&d.stage, t.stage.data(), t.n));
  TRY(dev_upload(&d.child_begin, t.child_begin.data(), t.n));
  TRY(dev_upload(&d.child_count, t.child_count.data(), t.n));
  TRY(dev_upload(&d.chain_off, t.chain_off.data(), t.chain_off.size()));
  TRY(dev_upload(&d.chain_node, t.chain_node.data(), t.chain_node.size()));
  TRY(dev_upload(&d.chain_parent, t.chain_parent.data(), t.chain_parent.size()));
  if (!t.top_nodes.empty()) TRY(dev_upload(&d.top_nodes, t.top_nodes.data(), t.top_nodes.size()));
  TRY(dev_upload(&d.top_expect, t.top_expect.data(), t.n));
  TRY(dev_upload(&d.path_off, t.path_off.data(), t.n + 1));
  if (!t.path_node.empty()) TRY(dev_upload(&d.path_node, t.path_node.data(), t.path_node.size()));
  TRY(dev_upload(&d.tree_of, t.tree_of.data(), t.n));
  TRY(dev_upload(&d.row, t.row.data(), t.n));
  TRY(dev_upload(&d.seg, t.seg.data(), t.seg.size()));
  TRY(dev_upload(&d.prob, t.prob.data(), t.n));
  TRY(dev_upload(&d.pbar, t.pbar.data(), t.n));
  return SMPC_OK;
}

}  // namespace

// smpc_factor_t is defined in smpc_internal.h

namespace {

IterArgs make_args(const smpc_factor_t* f) {
  const smpc_tree* t = f->tree;
  IterArgs a{};
  std::memset(&a, 0, sizeof a);
  a.n = f->n;
  a.n_x = f->n_x;
  a.n_u = f->n_u;
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
  a.packs = f->packs;
  a.pscale = f->pscale;
  a.pack_stride = f->pack_stride;
  a.ybuf0 = f->ybuf0;
  a.ybuf1 = f->ybuf1;
  a.wbuf = f->wbuf;
  a.h = f->h;
  a.uhat = f->uhat;
  a.e = f->e;
  a.beta = f->beta;
  a.spub = f->spub;
  a.rpub = f->rpub;
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
  a.cvec = f->cvec;
  a.theta = f->theta;
  a.xbar = a.ubar = nullptr;  // set by solves that keep the ergodic average
  a.res = f->res;
  a.counters = f->counters;
  a.flags = f->flags;
  a.wait_ns = f->wait_ns;
  a.R = f->R;
  a.res_tree = f->res_tree;  // NULL for a single tree
  a.tree_done = f->tree_done;
  return a;
}

// Upload float64 host values into a device buffer of the factor's vector type.
int put_vec(smpc_factor_t* f, void* dst, const double* src, size_t count, cudaStream_t s = nullptr) {
  if (count == 0) return SMPC_OK;
  if (f->prec == SMPC_FP64) {
    CK(cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyHostToDevice, s));
  } else {
    std::vector<float> tmp(count);
    for (size_t i = 0; i < count; ++i) tmp[i] = (float)src[i];
    CK(cudaMemcpyAsync(dst, tmp.data(), count * sizeof(float), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
  }
  return SMPC_OK;
}

// Upload float64 host values into a dual-state buffer (float64, or float32 pairs
// hi + lo with lo = 0 for values that are already float32).
int put_state(smpc_factor_t* f, void* dst, const double* src, size_t count) {
  if (count == 0) return SMPC_OK;
  if (f->prec == SMPC_FP64) {
    CK(cudaMemcpy(dst, src, count * sizeof(double), cudaMemcpyHostToDevice));
  } else {
    std::vector<float> tmp(2 * count);
    for (size_t i = 0; i < count; ++i) {
      const float hi = (float)src[i];
      tmp[2 * i] = hi;
      tmp[2 * i + 1] = (float)(src[i] - (double)hi);
    }
    CK(cudaMemcpy(dst, tmp.data(), tmp.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  return SMPC_OK;
}

int get_vec(const smpc_factor_t* f, double* dst, const void* src, size_t count) {
  if (count == 0) return SMPC_OK;
  if (f->prec == SMPC_FP64) {
    CK(cudaMemcpy(dst, src, count * sizeof(double), cudaMemcpyDeviceToHost));
  } else {
    std::vector<float> tmp(count);
    CK(cudaMemcpy(tmp.data(), src, count * sizeof(float), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < count; ++i) dst[i] = tmp[i];
  }
  return SMPC_OK;
}

int ensure_capacity(smpc_factor_t* f, int iters) {
  if (iters <= f->cap) return SMPC_OK;
  int cap = std::max(iters, 1024);
  unsigned long long* res = nullptr;
  double* cvec = nullptr;
  unsigned long long* res_tree = nullptr;
  TRY(f->alloc(&res, sizeof(unsigned long long) * 3 * (size_t)(cap + 2)));
  double* theta = nullptr;
  TRY(f->alloc(&cvec, sizeof(double) * (size_t)(cap + 2)));
  TRY(f->alloc(&theta, sizeof(double) * (size_t)(cap + 2)));
  if (f->R > 1) {  // forests: a residual per tree and iteration (each tree stops on its own)
    TRY(f->alloc(&res_tree, sizeof(unsigned long long) * 3 * (size_t)f->R * (size_t)(cap + 2)));
    CK(cudaMemset(res_tree, 0, sizeof(unsigned long long) * 3 * (size_t)f->R * (size_t)(cap + 2)));
  }
  f->drop_graphs();  // they hold the old buffers' addresses
  f->res = res;
  f->res_tree = res_tree;
  f->cvec = cvec;
  f->theta = theta;
  f->cap = cap;
  f->cvec_for = -1;
  return SMPC_OK;
}

// c_nu = theta_nu (1/theta_{nu-1} - 1) with theta_0 = theta_{-1} = 1 (eq. optim:theta:update),
// and theta_nu itself (the weights of the ergodic average, Sec. IV-A)
int upload_cvec(smpc_factor_t* f, int iters) {
  if (f->cvec_for >= iters) return SMPC_OK;
  std::vector<double> c(iters + 2), th(iters + 2);
  double tp = 1.0, t = 1.0;
  for (int nu = 0; nu < iters + 2; ++nu) {
    c[nu] = t * (1.0 / tp - 1.0);
    th[nu] = t;
    const double tn = 0.5 * (std::sqrt(t * t * t * t + 4.0 * t * t) - t * t);
    tp = t;
    t = tn;
  }
  CK(cudaMemcpy(f->cvec, c.data(), sizeof(double) * c.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(f->theta, th.data(), sizeof(double) * th.size(), cudaMemcpyHostToDevice));
  f->cvec_for = iters;
  return SMPC_OK;
}

uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// Largest eigenvalue of D^{1/2} H_D D^{1/2} by power iteration with the solve
// kernel in linear mode (the step arrays hold D).  Rayleigh quotient of the last step.
int power_iteration(smpc_factor_t* f, int iters, double* out) {
  const size_t ny = (size_t)f->n * f->nd;
  std::vector<double> y0(ny);
  uint64_t seed = 0x5eed5eed12345ull;
  double nrm = 0;
  for (size_t i = 0; i < ny; ++i) {
    double v = (double)(splitmix64(seed) >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
    if (f->prec != SMPC_FP64) v = (double)(float)v;
    y0[i] = v;
    nrm += v * v;
  }
  TRY(put_state(f, f->ybuf0, y0.data(), ny));
  double* pw = nullptr;
  TRY(f->alloc(&pw, sizeof(double) * 2 * (size_t)(iters + 2)));
  CK(cudaMemset(pw, 0, sizeof(double) * 2 * (size_t)(iters + 2)));
  CK(cudaMemcpy(pw, &nrm, sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemset(f->counters, 0, sizeof(int) * f->n));
  const int zero_flags[2] = {-1, 0};
  CK(cudaMemcpy(f->flags, zero_flags, sizeof zero_flags, cudaMemcpyHostToDevice));
  IterArgs a = make_args(f);
  a.pw = pw;
  a.pw_len = iters + 1;
  // one fixed schedule, so that the estimate does not depend on the autotuner's timing
  LaunchCfg cfg = iter_config(f->prec, a, f->num_sms, SCHED_CHAIN);
  if (cfg.stages < 1) cfg = iter_config(f->prec, a, f->num_sms, SCHED_NODE);
  if (cfg.stages < 1) {
    set_error("network too large for the shared-memory pipeline");
    return SMPC_ENOTSUP;
  }
  for (int k = 0; k < iters; ++k) {
    TRY(launch_iter(f->prec, a, cfg, k, MODE_BWD | MODE_LINEAR, nullptr));
    TRY(launch_iter(f->prec, a, cfg, k + 1, MODE_PROX | MODE_LINEAR, nullptr));
  }
  CK(cudaDeviceSynchronize());
  std::vector<double> h(2 * (size_t)(iters + 2));
  CK(cudaMemcpy(h.data(), pw, sizeof(double) * h.size(), cudaMemcpyDeviceToHost));
  int fl[2];
  CK(cudaMemcpy(fl, f->flags, sizeof fl, cudaMemcpyDeviceToHost));
  if (fl[1] != 0) {
    set_error("power iteration failed on the device (code %d)", fl[1]);
    return fl[1];
  }
  const int k = iters - 1;
  const double rq = h[a.pw_len + k] / std::sqrt(h[k]);
  if (!(std::isfinite(rq) && rq > 0)) {
    set_error("power iteration gave a non-positive Rayleigh quotient %g", rq);
    return SMPC_EDIVERGED;
  }
  *out = rq;
  return SMPC_OK;
}

}  // namespace

namespace smpc {

// Iteration schedule of a factor: the requested one, or (0) the fastest on this GPU,
// timed with CUDA events over a few solve-mode iterations of the factor's own tree and
// packs from a zero state; the state is cleared again afterwards.
int reset_state(smpc_factor_t* f);

int choose_schedule(smpc_factor_t* f, int requested) {
  if (requested < 0 || requested > kSchedules) {
    set_error("schedule must be 0 (auto), 1 (chain), 2 (node), 3 (hybrid) or 4 (fused chain pass)");
    return SMPC_EINVAL;
  }
  IterArgs a = make_args(f);
  const bool anchored = f->packs32 != nullptr;
  if (anchored) {
    a.ha = f->ha;
    a.wa = f->wa;
  }
  const int mode_extra = anchored ? MODE_DELTA : 0;
  bool fits[kSchedules + 1] = {};
  int n_fit = 0, only = SCHED_CHAIN;
  for (int s = 1; s <= kSchedules; ++s) {
    fits[s] = iter_config(f->prec, a, f->num_sms, s).stages > 0;
    if (fits[s]) {
      ++n_fit;
      only = s;
    }
  }
  if (requested != 0) {
    if (!fits[requested]) {
      set_error("the requested schedule does not fit this network");
      return SMPC_ENOTSUP;
    }
    f->schedule = requested;
    return SMPC_OK;
  }
  if (n_fit <= 1) {
    f->schedule = only;
    return SMPC_OK;
  }
  TRY(upload_cvec(f, 16));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = -1;
  constexpr int kWarm = 2, kTimed = 6;
  for (int s = 1; s <= kSchedules; ++s) {
    if (!fits[s]) continue;
    const LaunchCfg cfg = iter_config(f->prec, a, f->num_sms, s);
    int rc = SMPC_OK;
    for (int nu = 1; nu <= kWarm && !rc; ++nu) rc = launch_iter(f->prec, a, cfg, nu, MODE_BWD | MODE_PROX | mode_extra, nullptr);
    cudaEventRecord(e0);
    for (int nu = kWarm + 1; nu <= kWarm + kTimed && !rc; ++nu)
      rc = launch_iter(f->prec, a, cfg, nu, MODE_BWD | MODE_PROX | mode_extra, nullptr);
    cudaEventRecord(e1);
    float ms = 0;
    if (rc || cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (!rc) set_error("schedule timing failed: %s", cudaGetErrorString(cudaGetLastError()));
      return rc ? rc : SMPC_ECUDA;
    }
    if (best < 0 || ms < best) {
      best = ms;
      f->schedule = s;
    }
    f->tuned_ms[s] = ms / kTimed;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return reset_state(f);
}

// Back to the state a fresh factor has, after iterations run for timing.
int reset_state(smpc_factor_t* f) {
  const bool anchored = f->packs32 != nullptr;
  const size_t ny = (size_t)f->n * f->nd;
  const size_t nk = (size_t)f->n * f->n_k;
  if (cudaMemset(f->ybuf0, 0, ny * kStateSize) != cudaSuccess || cudaMemset(f->ybuf1, 0, ny * kStateSize) != cudaSuccess ||
      cudaMemset(f->wbuf, 0, nk * f->vs) != cudaSuccess || cudaMemset(f->h, 0, nk * f->vs) != cudaSuccess ||
      cudaMemset(f->counters, 0, sizeof(int) * f->n) != cudaSuccess ||
      cudaMemset(f->res, 0, sizeof(unsigned long long) * 3 * (size_t)(f->cap + 2)) != cudaSuccess ||
      (anchored && (cudaMemset(f->ha, 0, nk * sizeof(float)) != cudaSuccess ||
                    cudaMemset(f->wa, 0, nk * sizeof(float)) != cudaSuccess)) ||
      cudaDeviceSynchronize() != cudaSuccess) {
    set_error("schedule timing: %s", cudaGetErrorString(cudaGetLastError()));
    return SMPC_ECUDA;
  }
  return SMPC_OK;
}

// Width of the tensor-core GEMMs (nodes per MMA) of a bfloat16 shared-pack factor: the
// requested one, or (0) the fastest of 16, 32 and 64 nodes on this GPU, timed over a few
// delta iterations of the factor's schedule; the state is cleared again afterwards.
int tune_tc(smpc_factor_t* f, int requested) {
  IterArgs a = make_args(f);
  f->tc_width = 0;
  if (!f->packs32) return SMPC_OK;  // not a bfloat16 factor
  a.ha = f->ha;
  a.wa = f->wa;
  if (!iter_config(f->prec, a, f->num_sms, f->schedule).tc) return SMPC_OK;
  if (requested != 0) {
    if (requested != 16 && requested != 32 && requested != 64) {
      set_error("tc_width must be 0 (by timing), 16, 32 or 64");
      return SMPC_EINVAL;
    }
    f->tc_width = requested;
    return SMPC_OK;
  }
  TRY(upload_cvec(f, 16));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  constexpr int kWarm = 2, kTimed = 6;
  float best = -1;
  const int widths[3] = {16, 32, 64};
  for (int k = 0; k < 3; ++k) {
    const LaunchCfg cfg = iter_config(f->prec, a, f->num_sms, f->schedule, widths[k]);
    if (!cfg.tc || cfg.stages < 1) continue;
    int rc = SMPC_OK;
    const int mode = MODE_BWD | MODE_PROX | MODE_DELTA;
    for (int nu = 1; nu <= kWarm && !rc; ++nu) rc = launch_iter(f->prec, a, cfg, nu, mode, nullptr);
    cudaEventRecord(e0);
    for (int nu = kWarm + 1; nu <= kWarm + kTimed && !rc; ++nu) rc = launch_iter(f->prec, a, cfg, nu, mode, nullptr);
    cudaEventRecord(e1);
    float ms = 0;
    if (rc || cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (!rc) set_error("tensor-core width timing failed: %s", cudaGetErrorString(cudaGetLastError()));
      return rc ? rc : SMPC_ECUDA;
    }
    f->tc_ms[k] = ms / kTimed;
    if (best < 0 || ms < best) {
      best = ms;
      f->tc_width = widths[k];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return reset_state(f);
}

int plan_iters(const smpc_factor_t* f, const IterArgs& a, const smpc_solve_opts& opts, IterPlan* plan) {
  const int iters = opts.max_iters;
  if (opts.polish_iters < 0 || opts.polish_iters > iters || opts.anchor_every < 0) {
    set_error("polish_iters must be in [0, max_iters] and anchor_every >= 0");
    return SMPC_EINVAL;
  }
  plan->prec = f->prec;
  plan->args = a;
  plan->cfg = iter_config(f->prec, a, f->num_sms, f->schedule, f->tc_width);
  if (plan->cfg.stages < 1) {
    set_error("network too large for the shared-memory pipeline");
    return SMPC_ENOTSUP;
  }
  plan->polish_from = 0x7fffffff;
  plan->anchor_every = 0;
  plan->profile = f->profile;
  if (f->packs32) {  // SMPC_BF16: anchored solve, float32 packs for anchors and polish
    plan->args.ha = f->ha;
    plan->args.wa = f->wa;
    plan->args32 = plan->args;
    plan->args32.packs = f->packs32;
    plan->args32.pack_stride = f->pack_stride32;
    plan->cfg32 = iter_config(SMPC_FP32, plan->args32, f->num_sms, f->schedule);
    if (plan->cfg32.stages < 1) {
      set_error("network too large for the float32 pipeline");
      return SMPC_ENOTSUP;
    }
    plan->anchor_every = opts.anchor_every > 0 ? opts.anchor_every : 16;
    if (opts.polish_iters > 0) plan->polish_from = iters - opts.polish_iters;
  }
  return SMPC_OK;
}

int copy_final_y(smpc_factor_t* f, void* dst) {
  IterArgs a = make_args(f);
  TRY(launch_copy_final_y(f->prec, a, 0, dst, nullptr));
  CK(cudaStreamSynchronize(nullptr));
  return SMPC_OK;
}

// The iteration kernels' launch of iteration nu of a solve (the tail launch adds the
// last prox without a backward sweep).
int chunk_mode(int nu) { return MODE_BWD | MODE_CHECK | (nu > 0 ? MODE_PROX : 0); }

// Iterations [from, to) as one CUDA graph: captured from the planned launches on the
// factor's capture stream the first time this key is seen, then launched on s.  A
// capture or instantiation that fails turns graphs off for the factor and launches
// the chunk directly (the same kernels with the same arguments).
int launch_chunk_graph(smpc_factor_t* f, IterPlan& plan, int from, int to, const std::array<long long, 7>& key,
                       cudaStream_t s) {
  auto it = f->graphs.find(key);
  if (it == f->graphs.end()) {
    bool ok = true;
    if (!f->capture_stream && cudaStreamCreateWithFlags(&f->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
      ok = false;
    cudaGraph_t g = nullptr;
    const int k0 = plan.kernels;
    if (ok) ok = cudaStreamBeginCapture(f->capture_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      int rc = SMPC_OK;
      for (int nu = from; nu < to && rc == SMPC_OK; ++nu) rc = launch_planned(plan, nu, chunk_mode(nu), f->capture_stream);
      const cudaError_t e = cudaStreamEndCapture(f->capture_stream, &g);
      ok = rc == SMPC_OK && e == cudaSuccess && g != nullptr;
    }
    const int kernels = plan.kernels - k0;
    plan.kernels = k0;
    cudaGraphExec_t x = nullptr;
    if (ok) ok = cudaGraphInstantiate(&x, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();  // a refused capture leaves its error behind
    if (!ok) {
      f->graphs_off = true;
      for (int nu = from; nu < to; ++nu) TRY(launch_planned(plan, nu, chunk_mode(nu), s));
      return SMPC_OK;
    }
    it = f->graphs.emplace(key, smpc_factor_t::ChunkGraph{x, kernels}).first;
  }
  CK(cudaGraphLaunch(it->second.exec, s));
  plan.kernels += it->second.kernels;
  return SMPC_OK;
}

int launch_planned(IterPlan& plan, int nu, int mode, void* stream) {
  int prec = plan.prec;
  const IterArgs* a = &plan.args;
  LaunchCfg cfg = plan.cfg;
  bool anchor = false;
  if (plan.anchor_every > 0) {
    if (nu >= plan.polish_from || nu % plan.anchor_every == 0) {
      prec = SMPC_FP32;
      a = &plan.args32;
      cfg = plan.cfg32;
      mode |= MODE_ANCHOR;
      anchor = true;
    } else {
      mode |= MODE_DELTA;
    }
  }
  Profile* pf = plan.profile;
  const bool prof = pf && !anchor && (mode & MODE_BWD) && (mode & MODE_PROX) && nu >= 1 && pf->count < pf->capacity;
  if (prof) cfg.events = pf->ev.data() + (size_t)pf->count * Profile::kStageEvents;
  TRY(launch_iter(prec, *a, cfg, nu, mode, stream));
  plan.kernels += kernels_per_call(cfg, mode);
  if (prof) {
    pf->stages = kernels_per_call(cfg, mode);
    ++pf->count;
  }
  return SMPC_OK;
}

}  // namespace smpc

extern "C" {

int smpc_version(void) { return 1; }

const char* smpc_status_string(int s) {
  switch (s) {
    case SMPC_OK: return "ok";
    case SMPC_EINVAL: return "invalid argument";
    case SMPC_ENOMEM: return "out of memory";
    case SMPC_ECUDA: return "CUDA error";
    case SMPC_EBUSY: return "busy";
    case SMPC_ETIMEOUT: return "device wait timed out";
    case SMPC_EDIVERGED: return "diverged (non-finite iterates)";
    case SMPC_ENOTSUP: return "not supported";
    default: return "unknown status";
  }
}

const char* smpc_last_error(void) { return g_last_error.c_str(); }

int smpc_tree_create(int32_t n_nodes, const int32_t* parent, const double* prob, smpc_tree** out) {
  if (!out) {
    set_error("out is NULL");
    return SMPC_EINVAL;
  }
  *out = nullptr;
  smpc_tree* t = new (std::nothrow) smpc_tree();
  if (!t) return SMPC_ENOMEM;
  int rc = build_tree(n_nodes, parent, prob, *t);
  if (rc == SMPC_OK) rc = upload_tree(*t);
  if (rc != SMPC_OK) {
    free_tree_dev(t->dev);
    delete t;
    return rc;
  }
  *out = t;
  return SMPC_OK;
}

int smpc_tree_info_get(const smpc_tree* t, smpc_tree_info* info) {
  if (!t || !info) {
    set_error("NULL argument");
    return SMPC_EINVAL;
  }
  info->n_nodes = t->n;
  info->horizon = t->N;
  info->n_trees = t->R;
  info->n_leaves = t->n_leaves;
  info->n_chains = (int)t->chain_parent.size();
  info->n_top = (int)t->top_nodes.size();
  info->max_chain_len = t->max_chain_len;
  return SMPC_OK;
}

void smpc_tree_destroy(smpc_tree* t) {
  if (!t) return;
  free_tree_dev(t->dev);
  delete t;
}

int smpc_factor(const smpc_tree* tree, const smpc_network* net, const smpc_cost* cost,
                const smpc_factor_opts* opts, smpc_factor_t** out) {
  if (!out || !tree || !net || !cost) {
    set_error("NULL argument");
    return SMPC_EINVAL;
  }
  *out = nullptr;
  smpc_factor_opts o;
  std::memset(&o, 0, sizeof o);
  if (opts) o = *opts;
  if (o.precision < SMPC_FP64 || o.precision > SMPC_BF16) {
    set_error("unknown precision %d", o.precision);
    return SMPC_EINVAL;
  }
  const int n_x = net->n_x, n_u = net->n_u, n_d = net->n_d, n_e = net->n_e;
  if (n_x < 1 || n_u < 1 || n_d < 0 || n_e < 0 || !net->B || (n_d > 0 && !net->Gd) ||
      (n_e > 0 && (!net->E || (n_d > 0 && !net->Ed)))) {
    set_error("network sizes/pointers invalid");
    return SMPC_EINVAL;
  }
  if (!finite_array(net->B, (size_t)n_x * n_u) || (n_d && !finite_array(net->Gd, (size_t)n_x * n_d)) ||
      (n_e && !finite_array(net->E, (size_t)n_e * n_u)) || (n_e && n_d && !finite_array(net->Ed, (size_t)n_e * n_d))) {
    set_error("network matrices contain non-finite values");
    return SMPC_EINVAL;
  }
  bool general_A = false;  // A given and not the identity
  if (net->A) {
    if (!finite_array(net->A, (size_t)n_x * n_x)) {
      set_error("A contains non-finite values");
      return SMPC_EINVAL;
    }
    for (int i = 0; i < n_x; ++i)
      for (int j = 0; j < n_x; ++j)
        if (net->A[i * n_x + j] != (i == j ? 1.0 : 0.0)) general_A = true;
  }
  if (general_A && o.schedule != 0 && o.schedule != SCHED_NODE) {
    set_error("A != I runs on the node-parallel schedule (2) only");
    return SMPC_ENOTSUP;
  }
  if (!cost->alpha1 || !cost->W_u || !cost->x_min || !cost->x_max || !cost->x_s || !cost->u_min || !cost->u_max) {
    set_error("cost pointers must not be NULL");
    return SMPC_EINVAL;
  }
  if (!(cost->W_x >= 0) || !(cost->gamma_d >= 0) || !std::isfinite(cost->W_alpha) || !std::isfinite(cost->W_x) ||
      !std::isfinite(cost->gamma_d)) {
    set_error("W_x and gamma_d must be finite and non-negative");
    return SMPC_EINVAL;
  }
  for (int i = 0; i < n_x; ++i)
    if (!(cost->x_min[i] <= cost->x_max[i]) || !std::isfinite(cost->x_s[i])) {
      set_error("state bounds invalid at %d", i);
      return SMPC_EINVAL;
    }
  for (int i = 0; i < n_u; ++i)
    if (!(cost->u_min[i] <= cost->u_max[i])) {
      set_error("input bounds invalid at %d", i);
      return SMPC_EINVAL;
    }
  const bool explicit_steps = o.step_s || o.step_z || o.step_p;
  if (explicit_steps && !(o.step_s && o.step_z && o.step_p)) {
    set_error("explicit steps need step_s, step_z and step_p");
    return SMPC_EINVAL;
  }
  if (!(o.lambda >= 0) || !std::isfinite(o.lambda)) {
    set_error("lambda must be >= 0");
    return SMPC_EINVAL;
  }

  smpc_factor_t* f = new (std::nothrow) smpc_factor_t();
  if (!f) return SMPC_ENOMEM;
  auto fail = [&](int rc) {
    delete f;
    return rc;
  };
  f->tree = tree;
  f->prec = o.precision;
  f->n = tree->n;
  f->N = tree->rows;  // stage-indexed data rows: the sum of the trees' horizons
  f->R = tree->R;
  f->n_x = n_x;
  f->n_u = n_u;
  f->n_d = n_d;
  f->n_e = n_e;
  int rc = host_factor(*net, cost->W_u, f->hf);
  if (rc != SMPC_OK) return fail(rc);
  const int n_v = f->hf.n_v;
  f->n_v = n_v;
  f->n_k = n_x + n_u;
  f->nd = 2 * n_x + n_u;
  f->vs = vec_size(f->prec);
  f->ms = mat_size(f->prec);
  f->W_alpha = cost->W_alpha;
  f->gamma_d = cost->gamma_d;
  // Diagnostics: SMPC_PIPELINE_WAIT_NS (nanoseconds; 0 = one non-blocking test) replaces
  // the 2 s bound of node_mv's pack-pipeline waits for this factor's solves, so that a test
  // can make a wait give up (SMPC_ETIMEOUT) without a fault; the waits that let copies in
  // flight land keep the 2 s bound.
  if (const char* w = std::getenv("SMPC_PIPELINE_WAIT_NS")) {
    char* end = nullptr;
    const unsigned long long v = std::strtoull(w, &end, 10);
    if (end != w) f->wait_ns = v;
  }
  const int n = f->n, n_k = f->n_k, nd = f->nd;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&f->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    set_error("no CUDA device");
    return fail(SMPC_ECUDA);
  }
  // ---- shared float64 matrices on the device
  std::vector<double> K((size_t)n_k * n_v);
  for (int i = 0; i < n_x; ++i)
    for (int j = 0; j < n_v; ++j) K[(size_t)i * n_v + j] = f->hf.Bbar[(size_t)i * n_v + j];
  for (int i = 0; i < n_u; ++i)
    for (int j = 0; j < n_v; ++j) K[(size_t)(n_x + i) * n_v + j] = f->hf.L[(size_t)i * n_v + j];
  auto up64 = [&](double** dst, const double* src, size_t cnt) -> int {
    TRY(f->alloc(dst, cnt * sizeof(double)));
    if (cnt) CK(cudaMemcpy(*dst, src, cnt * sizeof(double), cudaMemcpyHostToDevice));
    return SMPC_OK;
  };
  if ((rc = up64(&f->K64, K.data(), K.size())) || (rc = up64(&f->Lam64, f->hf.Lam.data(), f->hf.Lam.size())) ||
      (rc = up64(&f->Pu, f->hf.Pu.data(), f->hf.Pu.size())) || (rc = up64(&f->Pe, f->hf.Pe.data(), f->hf.Pe.size())) ||
      (rc = up64(&f->Rhat, f->hf.Rhat.data(), f->hf.Rhat.size())) || (rc = up64(&f->L, f->hf.L.data(), f->hf.L.size())) ||
      (rc = up64(&f->alpha1, cost->alpha1, n_u)))
    return fail(rc);
  // ---- packs: one per node, or one shared pack (Lambda unscaled) and the node scales
  f->shared_packs = o.shared_packs != 0;
  const int np = f->shared_packs ? 1 : n;
  const double* pprob = f->shared_packs ? nullptr : tree->dev.prob;
  const long long pe = pack_entries(f->prec, n_k, n_v);
  f->pack_stride = f->shared_packs ? 0 : pe;
  if ((rc = f->alloc(&f->packs, (size_t)np * pe * f->ms))) return fail(rc);
  if ((rc = launch_pack(f->prec, np, n_k, n_v, f->K64, f->Lam64, pprob, f->packs, pe, nullptr))) return fail(rc);
  if (f->shared_packs) {
    std::vector<double> sc(n);
    for (int m = 0; m < n; ++m) sc[m] = 1.0 / (2.0 * tree->prob[m]);
    if ((rc = f->alloc(&f->pscale, (size_t)n * f->vs)) || (rc = put_vec(f, f->pscale, sc.data(), n))) return fail(rc);
  }
  if (f->prec == SMPC_BF16) {  // float32 packs for the anchor and polish iterations
    const long long pe32 = pack_entries(SMPC_FP32, n_k, n_v);
    f->pack_stride32 = f->shared_packs ? 0 : pe32;
    if ((rc = f->alloc(&f->packs32, (size_t)np * pe32 * sizeof(float)))) return fail(rc);
    if ((rc = launch_pack(SMPC_FP32, np, n_k, n_v, f->K64, f->Lam64, pprob, f->packs32, pe32, nullptr)))
      return fail(rc);
    const size_t hb = sizeof(float) * (size_t)n * n_k;
    if ((rc = f->alloc(&f->ha, hb)) || (rc = f->alloc(&f->wa, hb))) return fail(rc);
    if (cudaMemset(f->ha, 0, hb) != cudaSuccess || cudaMemset(f->wa, 0, hb) != cudaSuccess) return fail(SMPC_ECUDA);
  }
  // ---- vectors
  const size_t vs = f->vs;
  void** vecs[] = {&f->ybuf0, &f->ybuf1, &f->wbuf, &f->h, &f->uhat, &f->e, &f->beta, &f->spub, &f->rpub,
                   &f->uout, &f->xout, &f->step_s, &f->step_z, &f->step_p, &f->mu_s, &f->x_s, &f->x_min,
                   &f->x_max, &f->u_min, &f->u_max, &f->p0, &f->inv_s, &f->inv_z, &f->inv_p};
  const size_t cnts[] = {(size_t)n * nd, (size_t)n * nd, (size_t)n * n_k, (size_t)n * n_k, (size_t)n * n_u,
                         (size_t)n * n_x, (size_t)n * n_v, (size_t)n * n_x, (size_t)n * n_v, (size_t)n * n_u,
                         (size_t)n * n_x, (size_t)n, (size_t)n, (size_t)n * n_u, (size_t)n, (size_t)n_x,
                         (size_t)n_x, (size_t)n_x, (size_t)n_u, (size_t)n_u, (size_t)tree->R * n_x, (size_t)n,
                         (size_t)n, (size_t)n * n_u};
  static_assert(sizeof(vecs) / sizeof(vecs[0]) == sizeof(cnts) / sizeof(cnts[0]), "one count per vector");
  for (size_t i = 0; i < sizeof(cnts) / sizeof(cnts[0]); ++i) {
    const size_t bytes = cnts[i] * (i < 2 ? kStateSize : vs);  // the two dual buffers hold the state type
    if ((rc = f->alloc(vecs[i], bytes))) return fail(rc);
    if (cudaMemset(*vecs[i], 0, bytes) != cudaSuccess) {
      set_error("cudaMemset failed");
      return fail(SMPC_ECUDA);
    }
  }
  if (general_A && ((rc = f->alloc(&f->A, (size_t)n_x * n_x * vs)) || (rc = put_vec(f, f->A, net->A, (size_t)n_x * n_x))))
    return fail(rc);
  if ((rc = f->alloc(&f->uhat64, sizeof(double) * (size_t)n * n_u)) || (rc = f->alloc(&f->abar, sizeof(double) * (size_t)f->N * n_v)) ||
      (rc = f->alloc(&f->d_p, sizeof(double) * tree->R * n_x)) || (rc = f->alloc(&f->d_q, sizeof(double) * tree->R * n_u)) ||
      (rc = f->alloc(&f->d_dhat, sizeof(double) * (size_t)f->N * std::max(n_d, 1))) ||
      (rc = f->alloc(&f->d_eps, sizeof(double) * (size_t)n * std::max(n_d, 1))) ||
      (rc = f->alloc(&f->d_alpha2, sizeof(double) * (size_t)f->N * n_u)) || (rc = f->alloc(&f->counters, sizeof(int) * n)) ||
      (rc = f->alloc(&f->flags, sizeof(int) * 4)) || (rc = f->alloc(&f->tree_done, sizeof(int) * (size_t)f->R)))
    return fail(rc);
  if (cudaMemset(f->tree_done, 0xff, sizeof(int) * (size_t)f->R) != cudaSuccess) return fail(SMPC_ECUDA);
  if (cudaMemset(f->d_eps, 0, sizeof(double) * (size_t)n * std::max(n_d, 1)) != cudaSuccess ||
      cudaMemset(f->counters, 0, sizeof(int) * n) != cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void**>(&f->flags_host), sizeof(int) * 4) != cudaSuccess ||
      cudaEventCreateWithFlags(&f->ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&f->ev[1], cudaEventDisableTiming) != cudaSuccess) {
    set_error("device set-up failed: %s", cudaGetErrorString(cudaGetLastError()));
    return fail(SMPC_ECUDA);
  }
  {
    const int fl[4] = {0, 0, 0, 0};
    if (cudaMemcpy(f->flags, fl, sizeof fl, cudaMemcpyHostToDevice) != cudaSuccess) return fail(SMPC_ECUDA);
  }
  if ((rc = ensure_capacity(f, 1024))) return fail(rc);
  // bounds and safety weights
  std::vector<double> mu(n);
  for (int m = 0; m < n; ++m) mu[m] = cost->safety_unweighted ? cost->W_x : tree->prob[m] * cost->W_x;
  f->mu_host = mu;
  if ((rc = put_vec(f, f->mu_s, mu.data(), n)) || (rc = put_vec(f, f->x_s, cost->x_s, n_x)) ||
      (rc = put_vec(f, f->x_min, cost->x_min, n_x)) || (rc = put_vec(f, f->x_max, cost->x_max, n_x)) ||
      (rc = put_vec(f, f->u_min, cost->u_min, n_u)) || (rc = put_vec(f, f->u_max, cost->u_max, n_u)))
    return fail(rc);
  // ---- steps (Sec. IV-D)
  std::vector<double> ss(n), sz(n), sp((size_t)n * n_u);
  if (explicit_steps) {
    for (int m = 0; m < n; ++m) {
      ss[m] = o.step_s[m];
      sz[m] = o.step_z[m];
      if (!(ss[m] > 0 && sz[m] > 0)) {
        set_error("explicit steps must be positive");
        return fail(SMPC_EINVAL);
      }
    }
    for (size_t i = 0; i < sp.size(); ++i) {
      sp[i] = o.step_p[i];
      if (!(sp[i] > 0)) {
        set_error("explicit steps must be positive");
        return fail(SMPC_EINVAL);
      }
    }
    f->lambda = 0;
  } else {
    // Jacobi scaling: diagonal of the dual Hessian in closed form for A = I (with a general A
    // the same diagonal is used as the scaling: any positive diagonal is a valid preconditioner,
    // and lambda below comes from the scaled operator itself):
    //   x-blocks: diag(Bbar Rbar^-1 Bbar') * sum_{a in path(n)} k_a^2 / (2 p_a), k_a = path nodes from a to n
    //   inputs:   diag(L Rbar^-1 L') * sum_{a in path(n)} 1 / (2 p_a)
    // one scalar (mean) per distance block; zero-curvature inputs take their node's mean.
    double mB = 0;
    for (int i = 0; i < n_x; ++i) mB += f->hf.diagB[i];
    mB /= n_x;
    double dLmax = 0;
    for (int i = 0; i < n_u; ++i) dLmax = std::max(dLmax, f->hf.diagL[i]);
    for (int m = 0; m < n; ++m) {
      if (!o.precondition) {
        ss[m] = sz[m] = 1.0;
        for (int i = 0; i < n_u; ++i) sp[(size_t)m * n_u + i] = 1.0;
        continue;
      }
      std::vector<int> path;
      for (int k = m; k >= 0; k = tree->parent[k]) path.push_back(k);  // m .. root
      double cx = 0, cu = 0;
      for (size_t i = 0; i < path.size(); ++i) {
        const double k = (double)(i + 1);
        cx += k * k / (2.0 * tree->prob[path[i]]);
        cu += 1.0 / (2.0 * tree->prob[path[i]]);
      }
      ss[m] = sz[m] = 1.0 / (cx * mB);
      double live_sum = 0;
      int live = 0;
      for (int i = 0; i < n_u; ++i)
        if (f->hf.diagL[i] > 1e-12 * dLmax) {
          live_sum += f->hf.diagL[i];
          ++live;
        }
      const double fill = live ? live_sum / live : 1.0;
      for (int i = 0; i < n_u; ++i) {
        const double dl = f->hf.diagL[i] > 1e-12 * dLmax ? f->hf.diagL[i] : fill;
        sp[(size_t)m * n_u + i] = 1.0 / (cu * dl);
      }
    }
    double lam = o.lambda;
    if (lam <= 0) {
      if ((rc = put_vec(f, f->step_s, ss.data(), n)) || (rc = put_vec(f, f->step_z, sz.data(), n)) ||
          (rc = put_vec(f, f->step_p, sp.data(), sp.size())))
        return fail(rc);
      double L = 0;
      const int pit = o.power_iters > 0 ? o.power_iters : 200;
      if ((rc = power_iteration(f, pit, &L))) return fail(rc);
      const double margin = o.lambda_margin > 0 ? o.lambda_margin : 0.02;
      lam = 1.0 / (L * (1.0 + margin));
      // reset the buffers the power iteration used
      const size_t ny = (size_t)n * nd;
      if (cudaMemset(f->ybuf0, 0, ny * kStateSize) != cudaSuccess || cudaMemset(f->ybuf1, 0, ny * kStateSize) != cudaSuccess ||
          cudaMemset(f->counters, 0, sizeof(int) * n) != cudaSuccess)
        return fail(SMPC_ECUDA);
    }
    f->lambda = lam;
    for (auto& v : ss) v *= lam;
    for (auto& v : sz) v *= lam;
    for (auto& v : sp) v *= lam;
  }
  if ((rc = put_vec(f, f->step_s, ss.data(), n)) || (rc = put_vec(f, f->step_z, sz.data(), n)) ||
      (rc = put_vec(f, f->step_p, sp.data(), sp.size())))
    return fail(rc);
  {  // reciprocal steps: the prox turns y+ - w = lambda (x - t) into the residual x - t
    std::vector<double> is(n), iz(n), ip(sp.size());
    for (int m = 0; m < n; ++m) {
      is[m] = 1.0 / ss[m];
      iz[m] = 1.0 / sz[m];
    }
    for (size_t i = 0; i < sp.size(); ++i) ip[i] = 1.0 / sp[i];
    if ((rc = put_vec(f, f->inv_s, is.data(), n)) || (rc = put_vec(f, f->inv_z, iz.data(), n)) ||
        (rc = put_vec(f, f->inv_p, ip.data(), ip.size())))
      return fail(rc);
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    set_error("factor: %s", cudaGetErrorString(cudaGetLastError()));
    return fail(SMPC_ECUDA);
  }
  if ((rc = choose_schedule(f, o.schedule))) return fail(rc);
  if ((rc = tune_tc(f, o.tc_width))) return fail(rc);
  *out = f;
  return SMPC_OK;
}

void smpc_factor_destroy(smpc_factor_t* f) { delete f; }

size_t smpc_factor_device_bytes(const smpc_factor_t* f) { return f ? f->device_bytes : 0; }

int smpc_factor_schedule(const smpc_factor_t* f, double* ms_per_iter) {
  if (!f) {
    set_error("NULL factor");
    return -SMPC_EINVAL;
  }
  if (ms_per_iter) {
    ms_per_iter[0] = f->tuned_ms[SCHED_CHAIN];
    ms_per_iter[1] = f->tuned_ms[SCHED_NODE];
    ms_per_iter[2] = f->tuned_ms[SCHED_HYBRID];
    ms_per_iter[3] = f->tuned_ms[SCHED_FUSED];
  }
  return f->schedule;
}

int smpc_factor_tc_width(const smpc_factor_t* f, double* ms_per_width) {
  if (!f) {
    set_error("NULL factor");
    return -SMPC_EINVAL;
  }
  if (ms_per_width)
    for (int k = 0; k < 3; ++k) ms_per_width[k] = f->tc_ms[k];
  return f->tc_width;
}

int smpc_factor_steps(const smpc_factor_t* f, double* lambda, double* step_s, double* step_z, double* step_p) {
  if (!f) {
    set_error("NULL factor");
    return SMPC_EINVAL;
  }
  if (lambda) *lambda = f->lambda;
  if (step_s) TRY(get_vec(f, step_s, f->step_s, f->n));
  if (step_z) TRY(get_vec(f, step_z, f->step_z, f->n));
  if (step_p) TRY(get_vec(f, step_p, f->step_p, (size_t)f->n * f->n_u));
  return SMPC_OK;
}

}  // extern "C"

namespace smpc {
// Everything a solve does before its iteration chunks (Alg. 2 steps 1-3 up to the APG
// loop): checks, the launch plan, the step-data upload, the cost update of App. A, the
// initial duals and the per-solve flags, all enqueued on s.
int solve_begin(smpc_factor_t* f, const smpc_step_data* data, const smpc_solve_opts* opts, cudaStream_t s,
                IterPlan* plan_out, IterArgs* args_out) {
  if (!f || !data || !opts) {
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
  const int n = f->n, N = f->N, n_x = f->n_x, n_u = f->n_u, n_d = f->n_d;
  if (!finite_if_host(data->p, (size_t)f->R * n_x) || !finite_if_host(data->q, (size_t)f->R * n_u) ||
      !finite_if_host(data->alpha2, (size_t)N * n_u) ||
      (n_d && !finite_if_host(data->dhat, (size_t)N * n_d)) ||
      (data->eps && n_d && !finite_if_host(data->eps, (size_t)n * n_d))) {
    set_error("step data contains non-finite values");
    return SMPC_EINVAL;
  }
  const int iters = opts->max_iters;
  TRY(ensure_capacity(f, iters + 1));
  TRY(upload_cvec(f, iters + 1));
  // the launch plan (and its option checks) before any device work, so that a call
  // refused for its options leaves the factor's duals as they were
  IterArgs a = make_args(f);
  a.tol = opts->tol;
  if (opts->ergodic) {
    if (!f->xbar) TRY(f->alloc(&f->xbar, (size_t)n * n_x * f->vs));
    if (!f->ubar) TRY(f->alloc(&f->ubar, (size_t)n * n_u * f->vs));
    a.xbar = f->xbar;
    a.ubar = f->ubar;
  }
  IterPlan& plan = *plan_out;
  TRY(plan_iters(f, a, *opts, &plan));
  // step data -> device (Alg. 2 steps 1-2)
  CK(cudaMemcpyAsync(f->d_p, data->p, sizeof(double) * f->R * n_x, cudaMemcpyDefault, s));
  CK(cudaMemcpyAsync(f->d_q, data->q, sizeof(double) * f->R * n_u, cudaMemcpyDefault, s));
  if (n_d) CK(cudaMemcpyAsync(f->d_dhat, data->dhat, sizeof(double) * (size_t)N * n_d, cudaMemcpyDefault, s));
  if (data->eps && n_d)
    CK(cudaMemcpyAsync(f->d_eps, data->eps, sizeof(double) * (size_t)n * n_d, cudaMemcpyDefault, s));
  CK(cudaMemcpyAsync(f->d_alpha2, data->alpha2, sizeof(double) * (size_t)N * n_u, cudaMemcpyDefault, s));
  TRY(launch_convert(f->prec, f->d_p, f->p0, (long long)f->R * n_x, s));
  CostArgs c;
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
  TRY(launch_cost_update(f->prec, c, s));
  TRY(launch_init_duals(f->prec, a, (opts->warm_start && f->solved_once) ? 1 : 0, s));
  // arrival counters are reset by the CTAs that consume them; a solve that was cut
  // short by a device error may leave some behind
  CK(cudaMemsetAsync(f->counters, 0, sizeof(int) * (size_t)n, s));
  CK(cudaMemsetAsync(f->tree_done, 0xff, sizeof(int) * (size_t)f->R, s));  // after init_duals, which reads it
  if (f->res_tree)
    CK(cudaMemsetAsync(f->res_tree, 0, sizeof(unsigned long long) * 3 * (size_t)f->R * (size_t)(iters + 2), s));
  CK(cudaMemsetAsync(f->flags, 0xff, sizeof(int), s));
  CK(cudaMemsetAsync(f->flags + 1, 0, sizeof(int), s));
  CK(cudaMemsetAsync(f->res, 0, sizeof(unsigned long long) * 3 * (size_t)(iters + 2), s));
  *args_out = a;
  return SMPC_OK;
}

// After the iteration chunks: the last prox (the tail launch), the final dual and the
// outputs, enqueued on s; marks the factor's last solve.
int solve_end(smpc_factor_t* f, IterPlan& plan, const IterArgs& a, int launched, smpc_result* res, cudaStream_t s) {
  const int n = f->n, n_x = f->n_x, n_u = f->n_u;
  TRY(launch_planned(plan, launched, MODE_PROX | MODE_CHECK, s));
  TRY(launch_copy_final_y(f->prec, a, launched, res->y, s));
  if (res->u) CK(cudaMemcpyAsync(res->u, f->uout, (size_t)n * n_u * f->vs, cudaMemcpyDefault, s));
  if (res->x) CK(cudaMemcpyAsync(res->x, f->xout, (size_t)n * n_x * f->vs, cudaMemcpyDefault, s));
  if (res->ubar && a.ubar) CK(cudaMemcpyAsync(res->ubar, a.ubar, (size_t)n * n_u * f->vs, cudaMemcpyDefault, s));
  if (res->xbar && a.xbar) CK(cudaMemcpyAsync(res->xbar, a.xbar, (size_t)n * n_x * f->vs, cudaMemcpyDefault, s));
  f->solved_once = true;
  f->last_static = false;
  f->last_stream = s;
  f->last_launches = 6 + plan.kernels + 1;  // convert, 3 cost update, init, iterations and tail, final y
  res->launches = f->last_launches;
  res->iterations = -1;
  return SMPC_OK;
}
}  // namespace smpc

extern "C" {

int smpc_solve(smpc_factor_t* f, const smpc_step_data* data, const smpc_solve_opts* opts, smpc_result* res,
               void* stream) {
  if (!res) {
    set_error("NULL argument");
    return SMPC_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  IterPlan plan;
  IterArgs a;
  TRY(solve_begin(f, data, opts, s, &plan, &a));
  const int iters = opts->max_iters;
  const int chunk = opts->check_every > 0 ? opts->check_every : 128;
  int launched = 0, chunks = 0;
  bool stop = false;
  const bool graphs = opts->use_graph != 0 && !f->profile;
  long long tol_bits = 0;
  std::memcpy(&tol_bits, &opts->tol, sizeof tol_bits);
  while (launched < iters && !stop) {
    const int upto = std::min(iters, launched + chunk);
    if (graphs && !f->graphs_off) {
      TRY(launch_chunk_graph(f, plan, launched, upto, {launched, upto, iters, tol_bits, opts->polish_iters,
                                                       opts->anchor_every, opts->ergodic ? 1 : 0}, s));
    } else {
      for (int nu = launched; nu < upto; ++nu) TRY(launch_planned(plan, nu, chunk_mode(nu), s));
    }
    launched = upto;
    const int slot = chunks & 1;
    if (chunks >= 2) {  // the chunk two back has finished: look at its flags
      CK(cudaEventSynchronize(f->ev[slot]));
      if (f->flags_host[2 * slot] >= 0 || f->flags_host[2 * slot + 1] != 0) stop = true;
    }
    CK(cudaMemcpyAsync(f->flags_host + 2 * slot, f->flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(f->ev[slot], s));
    ++chunks;
  }
  TRY(solve_end(f, plan, a, launched, res, s));
  if (!opts->sync) return SMPC_OK;
  return smpc_solve_info(f, res);
}



int smpc_profile_solve(smpc_factor_t* f, const smpc_step_data* data, int32_t iters, double* stage_ms,
                       int32_t max_stages) {
  if (!f || !data || !stage_ms || max_stages < 1 || iters < 2 || iters > kProfileMaxIters) {
    set_error("smpc_profile_solve needs a factor, step data, 2 <= iters <= %d and room for the stage times",
              kProfileMaxIters);
    return -SMPC_EINVAL;
  }
  Profile P;
  P.capacity = iters;
  P.ev.assign((size_t)iters * Profile::kStageEvents, nullptr);
  auto release = [&]() {
    for (auto& e : P.ev)
      if (e) cudaEventDestroy(e);
  };
  for (auto& e : P.ev)
    if (cudaEventCreate(&e) != cudaSuccess) {
      set_error("cudaEventCreate failed");
      release();
      return -SMPC_ECUDA;
    }
  smpc_solve_opts o{};
  o.max_iters = iters;
  o.sync = 1;
  smpc_result r{};
  f->profile = &P;
  const int rc = smpc_solve(f, data, &o, &r, nullptr);
  f->profile = nullptr;
  if (rc != SMPC_OK || P.count == 0) {
    if (rc == SMPC_OK) set_error("no full iteration was profiled");
    release();
    return rc != SMPC_OK ? -rc : -SMPC_EINVAL;
  }
  std::vector<double> ms(P.stages, 0.0);
  for (int q = 0; q < P.count; ++q)
    for (int j = 0; j < P.stages; ++j) {
      float t = 0;
      cudaEvent_t* e = P.ev.data() + (size_t)q * Profile::kStageEvents;
      if (cudaEventElapsedTime(&t, e[j], e[j + 1]) != cudaSuccess) {
        set_error("cudaEventElapsedTime failed");
        release();
        return -SMPC_ECUDA;
      }
      ms[j] += t;
    }
  release();
  const int n = std::min(P.stages, (int)max_stages);
  for (int j = 0; j < n; ++j) stage_ms[j] = ms[j] / P.count;
  return P.stages;
}

int smpc_solve_trees(smpc_factor_t* f, int32_t* iterations, double* rho_rel) {
  if (!f || (!iterations && !rho_rel)) {
    set_error("NULL argument");
    return SMPC_EINVAL;
  }
  if (!f->solved_once) {
    set_error("no solve to report");
    return SMPC_EINVAL;
  }
  if (f->last_static) {
    set_error("the factor's last solve ran through smpc_solve_static, which keeps no per-tree record");
    return SMPC_EINVAL;
  }
  CK(cudaStreamSynchronize(f->last_stream));
  const int R = f->R;
  int fl[2];
  CK(cudaMemcpy(fl, f->flags, sizeof fl, cudaMemcpyDeviceToHost));
  std::vector<int> done(R, -1);
  CK(cudaMemcpy(done.data(), f->tree_done, sizeof(int) * R, cudaMemcpyDeviceToHost));
  for (int r = 0; r < R; ++r) {
    const int it = done[r] >= 0 ? done[r] : fl[0];
    if (iterations) iterations[r] = it;
    if (!rho_rel) continue;
    rho_rel[r] = 0;
    if (it < 1) continue;
    unsigned long long q[3];
    // a forest's own residual per tree; a single tree's is the solve's
    const unsigned long long* src = f->res_tree ? f->res_tree + 3 * ((size_t)(it - 1) * R + r)
                                                : f->res + 3 * (size_t)(it - 1);
    CK(cudaMemcpy(q, src, sizeof q, cudaMemcpyDeviceToHost));
    double v[3];
    std::memcpy(v, q, sizeof v);
    rho_rel[r] = v[0] / (1.0 + std::max(v[1], v[2]));
  }
  return SMPC_OK;
}

int smpc_solve_info(smpc_factor_t* f, smpc_result* res) {
  if (!f || !res) {
    set_error("NULL argument");
    return SMPC_EINVAL;
  }
  if (!f->solved_once) {
    set_error("no solve to complete");
    return SMPC_EINVAL;
  }
  if (f->last_static) {
    set_error("the factor's last solve ran through smpc_solve_static, whose host outputs come with opts->sync = 1");
    return SMPC_EINVAL;
  }
  const int n_u = f->n_u;
  CK(cudaStreamSynchronize(f->last_stream));
  res->launches = f->last_launches;
  int fl[2];
  CK(cudaMemcpy(fl, f->flags, sizeof fl, cudaMemcpyDeviceToHost));
  res->iterations = fl[0];
  if (fl[0] >= 1) {
    unsigned long long r3[3];
    CK(cudaMemcpy(r3, f->res + 3 * (size_t)(fl[0] - 1), sizeof r3, cudaMemcpyDeviceToHost));
    double v[3];
    std::memcpy(v, r3, sizeof v);
    res->rho = v[0];
    res->rho_rel = v[0] / (1.0 + std::max(v[1], v[2]));
  }
  if (res->history_host && fl[0] >= 1) {
    std::vector<unsigned long long> hist(3 * (size_t)fl[0]);
    CK(cudaMemcpy(hist.data(), f->res, sizeof(unsigned long long) * hist.size(), cudaMemcpyDeviceToHost));
    std::memcpy(res->history_host, hist.data(), sizeof(double) * hist.size());
  }
  if (res->u0_host) TRY(get_vec(f, res->u0_host, f->uout, (size_t)f->R * n_u));  // the roots are nodes 0..R-1
  if (fl[1] != 0) {
    set_error("solve failed on the device: %s", smpc_status_string(fl[1]));
    return fl[1];
  }
  return SMPC_OK;
}

}  // extern "C"
