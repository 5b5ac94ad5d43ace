// Shards: one scenario tree split over several GPUs (Sec. IV-B: the nodes of a stage are
// independent given their children's sums, so subtrees can be processed apart).
//
// The tree's chains (maximal leaf paths) are divided among the GPUs; the top nodes above
// them are replicated on every GPU.  One APG iteration of a shard is two halves around
// one exchange:
//   local: the forward sweep and prox of the shard's nodes (its chains and the top), and
//          the backward sweep along its own chains, which leaves each chain head's s and r;
//          then, per cut parent (a top node with chain children), the sums of s and r over
//          this GPU's heads below it;
//   -- the caller adds those sums over the GPUs (allreduce, sum) --
//   top:   the totals into the cut parents' chain children, then the backward sweep of the
//          top nodes, the same on every GPU.
// Every GPU then holds h for its chains and the whole top, which is all the next forward
// sweep of its nodes needs.  The residual of each iteration is a maximum over the GPUs:
// the caller takes the maximum of the three per-iteration entries over the GPUs (allreduce,
// max) before the next iteration's first launch reads it.

#include <algorithm>
#include <cstring>
#include <map>
#include <vector>

#include "smpc_internal.h"

using namespace smpc;

namespace {

#define SHCK(call)                                                                 \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      set_error("%s failed: %s", #call, cudaGetErrorString(e_));                   \
      return SMPC_ECUDA;                                                           \
    }                                                                              \
  } while (0)
#define SHTRY(expr)                 \
  do {                              \
    const int rc_ = (expr);         \
    if (rc_ != SMPC_OK) return rc_; \
  } while (0)

}  // namespace

struct smpc_shard {
  smpc_factor_t* f = nullptr;
  int c0 = 0, c1 = 0;
  int n_cut = 0, n_list = 0, n_top = 0;
  std::vector<int> cut_nodes;
  std::vector<int> nodes;  // the nodes this shard updates (host copy)
  int *d_cut_off = nullptr, *d_cut_heads = nullptr, *d_chl_off = nullptr, *d_chl = nullptr;
  int *d_nodes = nullptr, *d_seg = nullptr, *d_texp = nullptr;
  std::vector<void*> allocs;
  // the solve in progress
  bool begun = false;
  int iters = 0;
  cudaStream_t s = nullptr;
  IterArgs a{}, a_fp{}, a_chain{}, a_top{};
  LaunchCfg cfg_fp, cfg_chain, cfg_top;

  template <typename T>
  int upload(T** dst, const std::vector<T>& v) {
    const size_t bytes = std::max<size_t>(16, v.size() * sizeof(T));
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      set_error("cudaMalloc(%zu) failed", bytes);
      return SMPC_ENOMEM;
    }
    allocs.push_back(p);
    *dst = static_cast<T*>(p);
    if (!v.empty()) SHCK(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return SMPC_OK;
  }
  ~smpc_shard() {
    for (void* p : allocs) cudaFree(p);
  }
};

extern "C" {

int smpc_shard_create(smpc_factor_t* f, int32_t chain_begin, int32_t chain_end, smpc_shard** out) {
  if (!f || !out) {
    set_error("NULL argument");
    return SMPC_EINVAL;
  }
  *out = nullptr;
  const smpc_tree* t = f->tree;
  const int n_chains = (int)t->chain_parent.size(), n_top = (int)t->top_nodes.size();
  if (chain_begin < 0 || chain_end < chain_begin || chain_end > n_chains) {
    set_error("chain range [%d, %d) outside the tree's %d chains", chain_begin, chain_end, n_chains);
    return SMPC_EINVAL;
  }
  if (f->prec == SMPC_BF16) {
    set_error("shards run float64 and float32 factors (bfloat16 anchoring is not split)");
    return SMPC_ENOTSUP;
  }
  if (f->A) {
    set_error("shards run networks with A = I (the chain pass of a shard has no A' step)");
    return SMPC_ENOTSUP;
  }
  for (int c = 0; c < n_chains; ++c)
    if (t->chain_parent[c] < 0) {
      set_error("chain %d starts at a root: a tree split into shards needs top nodes above every chain", c);
      return SMPC_ENOTSUP;
    }
  auto* sh = new (std::nothrow) smpc_shard();
  if (!sh) {
    set_error("out of host memory");
    return SMPC_ENOMEM;
  }
  sh->f = f;
  sh->c0 = chain_begin;
  sh->c1 = chain_end;
  sh->n_top = n_top;
  // cut parents: the top nodes with chain children, in index order
  std::map<int, int> cut_index;
  for (int c = 0; c < n_chains; ++c) cut_index[t->chain_parent[c]] = 0;
  for (auto& kv : cut_index) {
    kv.second = (int)sh->cut_nodes.size();
    sh->cut_nodes.push_back(kv.first);
  }
  sh->n_cut = (int)sh->cut_nodes.size();
  // this shard's chain heads below each cut parent (CSR, heads in index order)
  std::vector<std::vector<int>> heads(sh->n_cut), chl(sh->n_cut);
  for (int c = chain_begin; c < chain_end; ++c) heads[cut_index[t->chain_parent[c]]].push_back(t->chain_node[t->chain_off[c]]);
  // every chain child of each cut parent (all shards), in index order
  for (int j = 0; j < sh->n_cut; ++j) {
    const int p = sh->cut_nodes[j];
    for (int c = t->child_begin[p]; c < t->child_begin[p] + t->child_count[p]; ++c)
      if (!t->is_top[c]) chl[j].push_back(c);
  }
  std::vector<int> cut_off(1, 0), cut_heads, chl_off(1, 0), chl_all;
  for (int j = 0; j < sh->n_cut; ++j) {
    for (int h : heads[j]) cut_heads.push_back(h);
    cut_off.push_back((int)cut_heads.size());
    for (int c : chl[j]) chl_all.push_back(c);
    chl_off.push_back((int)chl_all.size());
  }
  // the nodes this shard updates: the top and its own chains; its forward-sweep segments
  std::vector<int> nodes(t->top_nodes.begin(), t->top_nodes.end());
  for (int q = t->chain_off[chain_begin]; q < t->chain_off[chain_end]; ++q) nodes.push_back(t->chain_node[q]);
  std::sort(nodes.begin(), nodes.end());
  sh->n_list = (int)nodes.size();
  sh->nodes = nodes;
  std::vector<int> seg(t->seg.begin(), t->seg.begin() + (size_t)kSegInts * n_top);
  seg.insert(seg.end(), t->seg.begin() + (size_t)kSegInts * (n_top + chain_begin),
             t->seg.begin() + (size_t)kSegInts * (n_top + chain_end));
  // the top pass waits for each top node itself and its top children only
  std::vector<int> texp(t->n, 0);
  for (int q : t->top_nodes) {
    int k = 1;
    for (int c = t->child_begin[q]; c < t->child_begin[q] + t->child_count[q]; ++c) k += t->is_top[c] ? 1 : 0;
    texp[q] = k;
  }
  int rc = SMPC_OK;
  if ((rc = sh->upload(&sh->d_cut_off, cut_off)) || (rc = sh->upload(&sh->d_cut_heads, cut_heads)) ||
      (rc = sh->upload(&sh->d_chl_off, chl_off)) || (rc = sh->upload(&sh->d_chl, chl_all)) ||
      (rc = sh->upload(&sh->d_nodes, nodes)) || (rc = sh->upload(&sh->d_seg, seg)) ||
      (rc = sh->upload(&sh->d_texp, texp))) {
    delete sh;
    return rc;
  }
  *out = sh;
  return SMPC_OK;
}

void smpc_shard_destroy(smpc_shard* sh) { delete sh; }

int smpc_shard_info(const smpc_shard* sh, int32_t* n_cut, int32_t* width, int32_t* n_nodes) {
  if (!sh) {
    set_error("NULL shard");
    return SMPC_EINVAL;
  }
  if (n_cut) *n_cut = sh->n_cut;
  if (width) *width = sh->f->n_x + sh->f->n_v;
  if (n_nodes) *n_nodes = sh->n_list;
  return SMPC_OK;
}

int smpc_shard_nodes(const smpc_shard* sh, int32_t* nodes) {
  if (!sh || !nodes) {
    set_error("NULL argument");
    return SMPC_EINVAL;
  }
  std::copy(sh->nodes.begin(), sh->nodes.end(), nodes);
  return SMPC_OK;
}

int smpc_shard_begin(smpc_shard* sh, const smpc_step_data* data, const smpc_solve_opts* opts,
                     unsigned long long* residuals, void* stream) {
  if (!sh || !data || !opts || !residuals) {
    set_error("NULL argument");
    return SMPC_EINVAL;
  }
  smpc_factor_t* f = sh->f;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  IterPlan plan;
  IterArgs a;
  SHTRY(solve_begin(f, data, opts, s, &plan, &a));
  const smpc_tree* t = f->tree;
  sh->iters = opts->max_iters;
  sh->s = s;
  a.res = residuals;  // (rho, ||Hz||, ||t||) per iteration, maxima over every shard
  SHCK(cudaMemsetAsync(residuals, 0, sizeof(unsigned long long) * 3 * (size_t)(sh->iters + 2), s));
  sh->a = a;
  sh->a_fp = a;
  sh->a_fp.node_list = sh->d_nodes;
  sh->a_fp.n_list = sh->n_list;
  sh->a_fp.seg = sh->d_seg;
  sh->a_fp.n_chains = sh->c1 - sh->c0;
  sh->a_chain = a;
  sh->a_chain.chain_off = t->dev.chain_off + sh->c0;
  sh->a_chain.chain_parent = t->dev.chain_parent + sh->c0;
  sh->a_chain.n_chains = sh->c1 - sh->c0;
  sh->a_chain.n_top = 0;
  sh->a_top = a;
  sh->a_top.n_chains = 0;
  sh->a_top.top_expect = sh->d_texp;
  sh->cfg_fp = iter_config(f->prec, sh->a_fp, f->num_sms, SCHED_FUSED);
  sh->cfg_chain = iter_config(f->prec, sh->a_chain, f->num_sms, SCHED_CHAIN);
  sh->cfg_top = iter_config(f->prec, sh->a_top, f->num_sms, SCHED_CHAIN);
  sh->cfg_top.grid = std::max(1, std::min(sh->n_top, f->num_sms));
  if (sh->cfg_fp.stages < 1 || sh->cfg_chain.stages < 1 || sh->cfg_top.stages < 1) {
    set_error("network too large for the shared-memory pipeline");
    return SMPC_ENOTSUP;
  }
  sh->begun = true;
  return SMPC_OK;
}

int smpc_shard_step(smpc_shard* sh, int32_t nu, int32_t phase, void* exchange) {
  if (!sh || !sh->begun || nu < 0 || nu > sh->iters || (phase != 2 && !exchange)) {
    set_error("smpc_shard_step needs a begun shard, 0 <= nu <= max_iters and the exchange buffer");
    return SMPC_EINVAL;
  }
  smpc_factor_t* f = sh->f;
  const int prec = f->prec;
  cudaStream_t s = sh->s;
  if (phase == 0) {  // local half
    SHTRY(launch_iter(prec, sh->a_fp, sh->cfg_fp, nu, (nu >= 1 ? MODE_PROX : 0) | MODE_WONLY | MODE_CHECK, s));
    SHTRY(launch_iter(prec, sh->a_chain, sh->cfg_chain, nu, MODE_BWD | MODE_WREADY | MODE_NOCLIMB | MODE_CHECK, s));
    return launch_cut_sums(prec, sh->a, sh->n_cut, sh->d_cut_off, sh->d_cut_heads, exchange, s);
  }
  if (phase == 1) {  // top half, after the exchange
    SHTRY(launch_cut_scatter(prec, sh->a, sh->n_cut, sh->d_chl_off, sh->d_chl, exchange, s));
    return launch_iter(prec, sh->a_top, sh->cfg_top, nu, MODE_BWD | MODE_WREADY | MODE_CHECK, s);
  }
  if (phase == 2)  // the last forward sweep and prox (iteration nu - 1)
    return launch_iter(prec, sh->a_fp, sh->cfg_fp, nu, MODE_PROX | MODE_CHECK, s);
  set_error("phase must be 0 (local), 1 (top) or 2 (tail)");
  return SMPC_EINVAL;
}

int smpc_shard_finish(smpc_shard* sh, int32_t launched, smpc_result* res) {
  if (!sh || !sh->begun || !res) {
    set_error("smpc_shard_finish needs a begun shard and a result");
    return SMPC_EINVAL;
  }
  smpc_factor_t* f = sh->f;
  cudaStream_t s = sh->s;
  SHTRY(launch_copy_final_y(f->prec, sh->a, launched, res->y, s));
  if (res->u) SHCK(cudaMemcpyAsync(res->u, f->uout, (size_t)f->n * f->n_u * f->vs, cudaMemcpyDefault, s));
  if (res->x) SHCK(cudaMemcpyAsync(res->x, f->xout, (size_t)f->n * f->n_x * f->vs, cudaMemcpyDefault, s));
  SHCK(cudaStreamSynchronize(s));
  f->solved_once = true;
  f->last_static = true;  // its residuals live in the caller's buffer: smpc_solve_info does not apply
  f->last_stream = s;
  sh->begun = false;
  int fl[2];
  SHCK(cudaMemcpy(fl, f->flags, sizeof fl, cudaMemcpyDeviceToHost));
  res->iterations = fl[0];
  if (fl[0] >= 1) {
    unsigned long long r3[3];
    SHCK(cudaMemcpy(r3, sh->a.res + 3 * (size_t)(fl[0] - 1), sizeof r3, cudaMemcpyDeviceToHost));
    double v[3];
    std::memcpy(v, r3, sizeof v);
    res->rho = v[0];
    res->rho_rel = v[0] / (1.0 + std::max(v[1], v[2]));
  }
  if (fl[1] != 0) {
    set_error("solve failed on the device: %s", smpc_status_string(fl[1]));
    return fl[1];
  }
  return SMPC_OK;
}

int smpc_shard_flags(const smpc_shard* sh, int32_t* done, int32_t* error) {
  if (!sh || !done || !error) {
    set_error("NULL argument");
    return SMPC_EINVAL;
  }
  int fl[2];
  SHCK(cudaStreamSynchronize(sh->s));
  SHCK(cudaMemcpy(fl, sh->f->flags, sizeof fl, cudaMemcpyDeviceToHost));
  *done = fl[0];
  *error = fl[1];
  return SMPC_OK;
}

}  // extern "C"
