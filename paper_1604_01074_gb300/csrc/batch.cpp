// Batched solves: many scenario trees, on several networks, advanced together.
//
// A batch holds factors - each a single tree or a forest of trees on one network - and
// solves all of them with one launch per chunk of iterations: every chunk is one CUDA
// graph whose parallel branches are the factors' kernels for those iterations (the APG
// iteration of eq. apg-iteration with Algorithm 1 and the prox of App. C, per factor),
// so the trees of different networks share the GPU within each graph launch.  Each
// factor keeps its own state, step sizes and stop flags: a factor (or, in a forest, a
// tree) that met its tolerance leaves its iterates as they were, and its kernels in
// later chunks return at once.  The batch ends when every factor has stopped.

#include <array>
#include <cstring>
#include <map>
#include <vector>

#include "smpc_internal.h"

using namespace smpc;

namespace {

int chunk_mode(int nu) { return MODE_BWD | MODE_CHECK | (nu > 0 ? MODE_PROX : 0); }

#define BCK(call)                                                                  \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      set_error("%s failed: %s", #call, cudaGetErrorString(e_));                   \
      return SMPC_ECUDA;                                                           \
    }                                                                              \
  } while (0)
#define BTRY(expr)                  \
  do {                              \
    const int rc_ = (expr);         \
    if (rc_ != SMPC_OK) return rc_; \
  } while (0)

}  // namespace

struct smpc_batch {
  std::vector<smpc_factor_t*> f;
  std::vector<cudaStream_t> branch;  // one stream per factor: the branches of a chunk
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaStream_t capture = nullptr;
  int* flags_host = nullptr;  // pinned: 2 slots x factors x 2 ints
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    std::vector<int> kernels;  // per factor
  };
  // key: {first iteration, end, max_iters, tol bits, polish_iters, anchor_every, ergodic}
  std::map<std::array<long long, 7>, Graph> graphs;
  std::vector<const void*> bufs;  // the factors' iteration buffers the graphs were captured with
  bool graphs_off = false;

  void drop_graphs() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second.exec);
    graphs.clear();
  }
  ~smpc_batch() {
    drop_graphs();
    for (cudaStream_t s : branch) cudaStreamDestroy(s);
    for (cudaEvent_t e : join) cudaEventDestroy(e);
    if (fork) cudaEventDestroy(fork);
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
    if (capture) cudaStreamDestroy(capture);
    if (flags_host) cudaFreeHost(flags_host);
  }

  // iterations [from, to) of every factor, each on its branch stream between fork and join
  int enqueue(std::vector<IterPlan>& plan, int from, int to, cudaStream_t s) {
    BCK(cudaEventRecord(fork, s));
    for (size_t k = 0; k < f.size(); ++k) {
      BCK(cudaStreamWaitEvent(branch[k], fork, 0));
      for (int nu = from; nu < to; ++nu) BTRY(launch_planned(plan[k], nu, chunk_mode(nu), branch[k]));
      BCK(cudaEventRecord(join[k], branch[k]));
      BCK(cudaStreamWaitEvent(s, join[k], 0));
    }
    return SMPC_OK;
  }

  // one chunk as one graph launch (captured the first time this key is seen)
  int launch_chunk(std::vector<IterPlan>& plan, int from, int to, const std::array<long long, 7>& key,
                   cudaStream_t s) {
    auto it = graphs.find(key);
    if (it == graphs.end()) {
      std::vector<int> k0(f.size());
      for (size_t k = 0; k < f.size(); ++k) k0[k] = plan[k].kernels;
      bool ok = cudaStreamBeginCapture(capture, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      cudaGraph_t g = nullptr;
      if (ok) {
        const int rc = enqueue(plan, from, to, capture);
        const cudaError_t e = cudaStreamEndCapture(capture, &g);
        ok = rc == SMPC_OK && e == cudaSuccess && g != nullptr;
      }
      Graph G;
      for (size_t k = 0; k < f.size(); ++k) {
        G.kernels.push_back(plan[k].kernels - k0[k]);
        plan[k].kernels = k0[k];
      }
      if (ok) ok = cudaGraphInstantiate(&G.exec, g, 0) == cudaSuccess;
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();  // a refused capture leaves its error behind
      if (!ok) {  // plain launches from now on (same kernels, same arguments)
        graphs_off = true;
        return enqueue(plan, from, to, s);
      }
      it = graphs.emplace(key, std::move(G)).first;
    }
    BCK(cudaGraphLaunch(it->second.exec, s));
    for (size_t k = 0; k < f.size(); ++k) plan[k].kernels += it->second.kernels[k];
    return SMPC_OK;
  }
};

extern "C" {

int smpc_batch_create(int32_t count, smpc_factor_t* const* factors, smpc_batch** out) {
  if (!out || count < 1 || !factors) {
    set_error("smpc_batch_create needs count >= 1 factors and an output pointer");
    return SMPC_EINVAL;
  }
  *out = nullptr;
  for (int k = 0; k < count; ++k) {
    if (!factors[k]) {
      set_error("factor %d is NULL", k);
      return SMPC_EINVAL;
    }
    for (int j = 0; j < k; ++j)
      if (factors[j] == factors[k]) {
        set_error("factor %d appears twice in the batch", k);
        return SMPC_EINVAL;
      }
  }
  auto* b = new (std::nothrow) smpc_batch();
  if (!b) {
    set_error("out of host memory");
    return SMPC_ENOMEM;
  }
  b->f.assign(factors, factors + count);
  bool ok = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->ev[0], cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->ev[1], cudaEventDisableTiming) == cudaSuccess &&
            cudaMallocHost(reinterpret_cast<void**>(&b->flags_host), sizeof(int) * 4 * (size_t)count) == cudaSuccess;
  for (int k = 0; k < count && ok; ++k) {
    cudaStream_t st = nullptr;
    cudaEvent_t e = nullptr;
    ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (st) b->branch.push_back(st);
    if (e) b->join.push_back(e);
  }
  if (!ok) {
    set_error("batch set-up failed: %s", cudaGetErrorString(cudaGetLastError()));
    delete b;
    return SMPC_ECUDA;
  }
  *out = b;
  return SMPC_OK;
}

void smpc_batch_destroy(smpc_batch* b) { delete b; }

int smpc_batch_solve(smpc_batch* b, const smpc_step_data* data, const smpc_solve_opts* opts, smpc_result* res,
                     void* stream) {
  if (!b || !data || !opts || !res) {
    set_error("NULL argument");
    return SMPC_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t K = b->f.size();
  std::vector<IterPlan> plan(K);
  std::vector<IterArgs> args(K);
  for (size_t k = 0; k < K; ++k) BTRY(solve_begin(b->f[k], &data[k], opts, s, &plan[k], &args[k]));
  // graphs hold the factors' buffer addresses: a factor that grew its buffers drops them
  std::vector<const void*> bufs;
  for (smpc_factor_t* f : b->f) {
    bufs.push_back(f->res);
    bufs.push_back(f->cvec);
  }
  if (bufs != b->bufs) {
    b->drop_graphs();
    b->bufs = bufs;
  }
  const int iters = opts->max_iters;
  const int chunk = opts->check_every > 0 ? opts->check_every : 128;
  const bool graphs = opts->use_graph != 0;
  long long tol_bits = 0;
  std::memcpy(&tol_bits, &opts->tol, sizeof tol_bits);
  int launched = 0, chunks = 0;
  bool stop = false;
  while (launched < iters && !stop) {
    const int upto = std::min(iters, launched + chunk);
    if (graphs && !b->graphs_off)
      BTRY(b->launch_chunk(plan, launched, upto, {launched, upto, iters, tol_bits, opts->polish_iters,
                                                  opts->anchor_every, opts->ergodic ? 1 : 0}, s));
    else
      BTRY(b->enqueue(plan, launched, upto, s));
    launched = upto;
    const int slot = chunks & 1;
    int* fh = b->flags_host + 2 * K * slot;
    if (chunks >= 2) {  // the chunk two back has finished: every factor stopped?
      BCK(cudaEventSynchronize(b->ev[slot]));
      bool all = true;
      for (size_t k = 0; k < K; ++k) all = all && (fh[2 * k] >= 0 || fh[2 * k + 1] != 0);
      stop = all;
    }
    for (size_t k = 0; k < K; ++k)
      BCK(cudaMemcpyAsync(fh + 2 * k, b->f[k]->flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    BCK(cudaEventRecord(b->ev[slot], s));
    ++chunks;
  }
  for (size_t k = 0; k < K; ++k) BTRY(solve_end(b->f[k], plan[k], args[k], launched, &res[k], s));
  if (!opts->sync) return SMPC_OK;
  int first = SMPC_OK;
  for (size_t k = 0; k < K; ++k) {
    const int rc = smpc_solve_info(b->f[k], &res[k]);
    if (rc != SMPC_OK && first == SMPC_OK) first = rc;
  }
  return first;
}

}  // extern "C"
