// Serving: continuous batching of SMPC solves on one GPU (smpc_server_*).
//
// A closed-loop controller solves one SMPC problem per sampling period (Alg. 2);
// a service runs many controllers - trees of different sizes - against one GPU.
// Requests are queued by smpc_submit and admitted into execution slots as slots
// and device memory free up.  Each slot is a worker thread driving smpc_solve on
// its own non-blocking CUDA stream, so the kernels of admitted solves overlap on
// the device while new requests keep arriving.  Admission is by HBM footprint: a
// request is admitted when the device memory of the factors being solved, plus its
// own factor's, fits the server's budget.  A factor is held from admission until
// its ticket is polled, so the duals it keeps for warm starts and the outputs
// smpc_poll copies belong to one request at a time.

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "smpc_internal.h"

using namespace smpc;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  smpc_factor_t* f = nullptr;
  std::vector<double> p, q, dhat, eps, alpha2;
  bool has_eps = false;
  smpc_solve_opts opts{};
  size_t admitted_bytes = 0;  // the factor's footprint counted at admission (a solve may grow it)
  // results
  bool done = false;
  int status = SMPC_OK;
  std::string error;
  int iterations = 0, launches = 0;
  double rho = 0, rho_rel = 0;
  std::vector<double> u0, history;
  Clock::time_point t_submit, t_start, t_end;
};

// Copies `count` doubles from host or device memory.
int copy_in(std::vector<double>& dst, const double* src, size_t count) {
  dst.resize(count);
  if (count == 0) return SMPC_OK;
  cudaPointerAttributes at{};
  const bool dev = cudaPointerGetAttributes(&at, src) == cudaSuccess && at.type == cudaMemoryTypeDevice;
  cudaGetLastError();
  if (dev) {
    if (cudaMemcpy(dst.data(), src, count * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
      set_error("copying device step data failed");
      return SMPC_ECUDA;
    }
  } else {
    std::memcpy(dst.data(), src, count * sizeof(double));
  }
  return SMPC_OK;
}

}  // namespace

struct smpc_server {
  size_t budget = 0;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  uint64_t next_ticket = 1;
  std::deque<Request*> queue;                        // submitted, not admitted (arrival order)
  std::unordered_map<uint64_t, Request*> tickets;    // every request not yet returned by smpc_poll
  std::unordered_set<smpc_factor_t*> held;           // factors admitted and not yet polled
  size_t in_flight_bytes = 0;                        // device bytes of the factors being solved
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;

  void worker(int slot);
  Request* pick_locked();
};

Request* smpc_server::pick_locked() {
  for (auto it = queue.begin(); it != queue.end(); ++it) {
    Request* r = *it;
    if (held.count(r->f)) continue;  // an earlier request of this factor is running or unpolled
    if (in_flight_bytes + r->f->device_bytes > budget) continue;
    queue.erase(it);
    held.insert(r->f);
    r->admitted_bytes = r->f->device_bytes;
    in_flight_bytes += r->admitted_bytes;
    return r;
  }
  return nullptr;
}

void smpc_server::worker(int slot) {
  cudaSetDevice(device);
  cudaStream_t s = streams[slot];
  // pinned staging of the step data, so that the uploads run asynchronously on the slot's stream
  std::vector<double*> pin(5, nullptr);
  std::vector<size_t> cap(5, 0);
  auto stage = [&](int k, const std::vector<double>& v) -> const double* {
    if (v.empty()) return nullptr;
    if (cap[k] < v.size()) {
      if (pin[k]) cudaFreeHost(pin[k]);
      pin[k] = nullptr;
      cap[k] = 0;
      if (cudaMallocHost(reinterpret_cast<void**>(&pin[k]), v.size() * sizeof(double)) != cudaSuccess) return nullptr;
      cap[k] = v.size();
    }
    std::memcpy(pin[k], v.data(), v.size() * sizeof(double));
    return pin[k];
  };
  std::unique_lock<std::mutex> lk(mu);
  while (true) {
    Request* r = nullptr;
    cv.wait(lk, [&] { return stop || (r = pick_locked()) != nullptr; });
    if (!r) break;  // stopping
    lk.unlock();
    r->t_start = Clock::now();
    smpc_step_data d{};
    d.p = stage(0, r->p);
    d.q = stage(1, r->q);
    d.dhat = stage(2, r->dhat);
    d.eps = r->has_eps ? stage(3, r->eps) : nullptr;
    d.alpha2 = stage(4, r->alpha2);
    bool host_ok = true;  // no exception leaves the worker: a failed allocation is the request's status
    try {
      r->u0.assign((size_t)r->f->R * r->f->n_u, 0.0);
      r->history.assign((size_t)r->opts.max_iters * 3, 0.0);
    } catch (const std::bad_alloc&) {
      host_ok = false;
    }
    smpc_result res{};
    res.u0_host = r->u0.data();
    res.history_host = r->history.data();
    smpc_solve_opts o = r->opts;
    o.sync = 1;  // this worker waits; the other slots keep running
    int rc = SMPC_OK;
    if (!host_ok) {
      rc = SMPC_ENOMEM;
      r->error = "host allocation of the residual history failed";
    } else if ((r->p.size() && !d.p) || (r->alpha2.size() && !d.alpha2)) {
      rc = SMPC_ENOMEM;
      r->error = "pinned staging allocation failed";
    } else {
      rc = smpc_solve(r->f, &d, &o, &res, s);
      if (rc != SMPC_OK) r->error = smpc_last_error();
    }
    r->t_end = Clock::now();
    lk.lock();
    r->status = rc;
    r->iterations = res.iterations;
    r->rho = res.rho;
    r->rho_rel = res.rho_rel;
    r->launches = res.launches;
    r->done = true;
    // exactly what admission added: the solve may have grown the factor's iteration buffers
    // (the factor stays held until the ticket is polled)
    in_flight_bytes -= r->admitted_bytes;
    cv.notify_all();
  }
  lk.unlock();
  for (double* p : pin)
    if (p) cudaFreeHost(p);
}

extern "C" {

int smpc_server_create(size_t hbm_budget, int32_t max_slots, smpc_server** out) {
  if (!out || max_slots < 1 || hbm_budget == 0) {
    set_error("smpc_server_create needs hbm_budget > 0, max_slots >= 1 and an output pointer");
    return SMPC_EINVAL;
  }
  *out = nullptr;
  auto* sv = new (std::nothrow) smpc_server();
  if (!sv) {
    set_error("out of host memory");
    return SMPC_ENOMEM;
  }
  sv->budget = hbm_budget;
  if (cudaGetDevice(&sv->device) != cudaSuccess) {
    delete sv;
    set_error("no CUDA device");
    return SMPC_ECUDA;
  }
  for (int k = 0; k < max_slots; ++k) {
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      for (cudaStream_t t : sv->streams) cudaStreamDestroy(t);
      delete sv;
      set_error("cudaStreamCreate failed");
      return SMPC_ECUDA;
    }
    sv->streams.push_back(s);
  }
  for (int k = 0; k < max_slots; ++k) sv->workers.emplace_back([sv, k] { sv->worker(k); });
  *out = sv;
  return SMPC_OK;
}

void smpc_server_destroy(smpc_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv.notify_all();
  for (auto& t : sv->workers) t.join();  // solves already admitted finish first
  for (cudaStream_t s : sv->streams) cudaStreamDestroy(s);
  for (auto& kv : sv->tickets) delete kv.second;
  delete sv;
}

int smpc_submit(smpc_server* sv, smpc_factor_t* f, const smpc_step_data* data, const smpc_solve_opts* opts,
                uint64_t* ticket) {
  if (!sv || !f || !data || !opts || !ticket) {
    set_error("NULL argument");
    return SMPC_EINVAL;
  }
  if (!data->p || !data->q || !data->alpha2 || (f->n_d > 0 && !data->dhat) || opts->max_iters < 1 ||
      opts->max_iters > SMPC_MAX_ITERS || !(opts->tol >= 0)) {
    set_error("step data needs p, q, dhat and alpha2; max_iters in [1, %d] and tol >= 0", SMPC_MAX_ITERS);
    return SMPC_EINVAL;
  }
  if (f->device_bytes > sv->budget) {
    set_error("the factor needs %zu bytes of device memory; the server's budget is %zu bytes", f->device_bytes,
              sv->budget);
    return SMPC_EBUSY;
  }
  auto* r = new (std::nothrow) Request();
  if (!r) {
    set_error("out of host memory");
    return SMPC_ENOMEM;
  }
  r->f = f;
  r->opts = *opts;
  int rc = SMPC_OK;
  if ((rc = copy_in(r->p, data->p, (size_t)f->R * f->n_x)) || (rc = copy_in(r->q, data->q, (size_t)f->R * f->n_u)) ||
      (rc = copy_in(r->alpha2, data->alpha2, (size_t)f->N * f->n_u)) ||
      (f->n_d && (rc = copy_in(r->dhat, data->dhat, (size_t)f->N * f->n_d))) ||
      (data->eps && f->n_d && (rc = copy_in(r->eps, data->eps, (size_t)f->n * f->n_d)))) {
    delete r;
    return rc;
  }
  r->has_eps = data->eps != nullptr && f->n_d > 0;
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    r->ticket = sv->next_ticket++;
    sv->tickets[r->ticket] = r;
    sv->queue.push_back(r);
  }
  sv->cv.notify_all();
  *ticket = r->ticket;
  return SMPC_OK;
}

int smpc_poll(smpc_server* sv, uint64_t ticket, smpc_result* res, int32_t* done) {
  if (!sv || !done) {
    set_error("NULL argument");
    return SMPC_EINVAL;
  }
  Request* r = nullptr;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->tickets.find(ticket);
    if (it == sv->tickets.end()) {
      set_error("unknown ticket %llu", (unsigned long long)ticket);
      return SMPC_EINVAL;
    }
    r = it->second;
    if (!r->done) {
      *done = 0;
      return SMPC_OK;
    }
  }
  *done = 1;
  int rc = r->status;
  if (rc != SMPC_OK) {
    set_error("%s", r->error.c_str());
  } else if (res) {
    res->iterations = r->iterations;
    res->rho = r->rho;
    res->rho_rel = r->rho_rel;
    res->launches = r->launches;
    res->queue_ms = std::chrono::duration<double, std::milli>(r->t_start - r->t_submit).count();
    res->run_ms = std::chrono::duration<double, std::milli>(r->t_end - r->t_start).count();
    if (res->u0_host) std::memcpy(res->u0_host, r->u0.data(), r->u0.size() * sizeof(double));
    if (res->history_host && r->iterations > 0)
      std::memcpy(res->history_host, r->history.data(), (size_t)r->iterations * 3 * sizeof(double));
    // the factor is still held by this ticket: its buffers hold this solve's iterates
    smpc_factor_t* f = r->f;
    const size_t vs = f->vs;
    if (res->u && cudaMemcpy(res->u, f->uout, (size_t)f->n * f->n_u * vs, cudaMemcpyDefault) != cudaSuccess) rc = SMPC_ECUDA;
    if (res->x && cudaMemcpy(res->x, f->xout, (size_t)f->n * f->n_x * vs, cudaMemcpyDefault) != cudaSuccess) rc = SMPC_ECUDA;
    if (res->y && rc == SMPC_OK) rc = copy_final_y(f, res->y);
    if (r->opts.ergodic && f->ubar && res->ubar &&
        cudaMemcpy(res->ubar, f->ubar, (size_t)f->n * f->n_u * vs, cudaMemcpyDefault) != cudaSuccess)
      rc = SMPC_ECUDA;
    if (r->opts.ergodic && f->xbar && res->xbar &&
        cudaMemcpy(res->xbar, f->xbar, (size_t)f->n * f->n_x * vs, cudaMemcpyDefault) != cudaSuccess)
      rc = SMPC_ECUDA;
    if (rc == SMPC_ECUDA) set_error("copying the outputs of ticket %llu failed", (unsigned long long)ticket);
  }
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->held.erase(r->f);
    sv->tickets.erase(ticket);
  }
  sv->cv.notify_all();
  delete r;
  return rc;
}

}  // extern "C"
