// Device code of the APG solver for scenario-tree stochastic MPC (sm_103a).
//
// One launch of `apg_iter` = one APG iteration (eq. apg-iteration):
//   Phase P (MODE_PROX) finishes iteration nu-1: the forward sweep of Algorithm 1
//     as prefix sums over the tree of h = [Bbar; L] delta (written by the previous
//     launch), the prox of g (App. C) block by block, the dual update, and the
//     extrapolation w^nu of the next iteration (eq. optim:acceleration);
//   Phase B (MODE_BWD) runs the backward sweep of Algorithm 1 for iteration nu.
// The tree is split into "chains" (maximal leaf paths: every node of a chain has
// at most one child) and "top" nodes (everything else).  CTA b owns chains
// b, b + G, ...; it streams each chain node's pack [Bbar; L | Lambda/(2 p_n)]
// through shared memory with cp.async.bulk (mbarrier completion), so every matrix
// entry is read from HBM once per iteration.  Top nodes are reduced without any
// barrier: each top node counts arrivals (its children, plus its own Phase P) and
// the CTA that arrives last processes it (reading its pack straight from global
// memory), then arrives at its parent.  No CTA ever waits for another CTA.
//
// Backward sweep at node n (A = I; Algorithm 1 with Phi s + Psi psi + Lambda sigma
// regrouped as Lambda r, since Phi = Lambda Bbar' and Psi = Lambda L'):
//   s_n = xi_n + sum_c s_c,   r_n = beta_n + sum_c r_c + [Bbar; L]' [s_n; psi_n],
//   delta_n = Lambda r_n / (2 p_n),   h_n = [Bbar; L] delta_n.
// Forward sweep: v_n = v_pi + delta_n gives L v_n = sum over the path of L delta
// and Bbar v_n = sum over the path of Bbar delta, so u_n = u_hat_n + sum_path h^u
// and x_n = x_pi + Bbar v_n + e_n with x_pi(root) = p.

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "smpc_internal.h"

namespace smpc {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kChunk = 16384;            // bytes per bulk copy instruction
constexpr uint64_t kWaitNs = 2000000000ull;  // bounded mbarrier wait: 2 s

__device__ __forceinline__ double to_acc(double v) { return v; }
__device__ __forceinline__ float to_acc(float v) { return v; }
__device__ __forceinline__ float to_acc(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename MT>
struct Acc;
template <>
struct Acc<double> { using T = double; };
template <>
struct Acc<float> { using T = float; };
template <>
struct Acc<__nv_bfloat16> { using T = float; };

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(b))
      : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for phase `parity` of barrier b; gives up after kWaitNs and returns false.
__device__ bool mbar_wait(uint64_t* b, uint32_t parity) {
  if (mbar_test(b, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_test(b, parity)) {
    if (global_ns() - t0 > kWaitNs) return false;
  }
  return true;
}

template <typename T>
__device__ __forceinline__ T ldcg(const T* p) {
  return *reinterpret_cast<const volatile T*>(p);
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* slot, double v) {
  if (!(v >= 0.0)) v = __longlong_as_double(0x7ff0000000000000ll);  // NaN -> +inf
  atomicMax(slot, static_cast<unsigned long long>(__double_as_longlong(v)));
}

template <typename AT>
__device__ __forceinline__ AT warp_sum(AT v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ------------------------------------------------------------------ CTA mat-vecs
// out[j] = sum_i A[i*C + j] x[i] for j < C (A' x), A row-major R x C.
template <typename MT, typename AT>
__device__ void matvec_t(const MT* A, int R, int C, const AT* x, AT* out, AT* part) {
  const int t = threadIdx.x;
  if (C >= kThreads / 2) {
    for (int j = t; j < C; j += kThreads) {
      AT a0 = 0, a1 = 0, a2 = 0, a3 = 0;
      int i = 0;
      for (; i + 3 < R; i += 4) {
        a0 += to_acc(A[(i + 0) * C + j]) * x[i + 0];
        a1 += to_acc(A[(i + 1) * C + j]) * x[i + 1];
        a2 += to_acc(A[(i + 2) * C + j]) * x[i + 2];
        a3 += to_acc(A[(i + 3) * C + j]) * x[i + 3];
      }
      for (; i < R; ++i) a0 += to_acc(A[i * C + j]) * x[i];
      out[j] = (a0 + a1) + (a2 + a3);
    }
    __syncthreads();
    return;
  }
  int P = kThreads / C;
  if (P > 8) P = 8;
  const int rc = (R + P - 1) / P;
  if (t < P * C) {
    const int j = t % C, p = t / C;
    const int i0 = p * rc, i1 = min(R, i0 + rc);
    AT a0 = 0, a1 = 0;
    int i = i0;
    for (; i + 1 < i1; i += 2) {
      a0 += to_acc(A[i * C + j]) * x[i];
      a1 += to_acc(A[(i + 1) * C + j]) * x[i + 1];
    }
    if (i < i1) a0 += to_acc(A[i * C + j]) * x[i];
    part[p * C + j] = a0 + a1;
  }
  __syncthreads();
  for (int j = t; j < C; j += kThreads) {
    AT s = 0;
    for (int p = 0; p < P; ++p) s += part[p * C + j];
    out[j] = s;
  }
  __syncthreads();
}

// out[i] = sum_j A[i*C + j] x[j] for i < R (A x).
template <typename MT, typename AT>
__device__ void matvec_n(const MT* A, int R, int C, const AT* x, AT* out, AT* part) {
  const int t = threadIdx.x;
  if (R >= kThreads / 2) {
    for (int i = t; i < R; i += kThreads) {
      const MT* row = A + (long long)i * C;
      AT a0 = 0, a1 = 0, a2 = 0, a3 = 0;
      int j = 0;
      for (; j + 3 < C; j += 4) {
        a0 += to_acc(row[j + 0]) * x[j + 0];
        a1 += to_acc(row[j + 1]) * x[j + 1];
        a2 += to_acc(row[j + 2]) * x[j + 2];
        a3 += to_acc(row[j + 3]) * x[j + 3];
      }
      for (; j < C; ++j) a0 += to_acc(row[j]) * x[j];
      out[i] = (a0 + a1) + (a2 + a3);
    }
    __syncthreads();
    return;
  }
  int P = kThreads / R;
  if (P > 8) P = 8;
  const int cc = (C + P - 1) / P;
  if (t < P * R) {
    const int i = t % R, p = t / R;
    const int j0 = p * cc, j1 = min(C, j0 + cc);
    AT a0 = 0;
    for (int j = j0; j < j1; ++j) a0 += to_acc(A[(long long)i * C + j]) * x[j];
    part[p * R + i] = a0;
  }
  __syncthreads();
  for (int i = t; i < R; i += kThreads) {
    AT s = 0;
    for (int p = 0; p < P; ++p) s += part[p * R + i];
    out[i] = s;
  }
  __syncthreads();
}

// ------------------------------------------------------------------ kernel state
template <typename MT>
struct Smem {
  MT* K[4];
  MT* Lm[4];
  uint64_t* barK;
  uint64_t* barL;
  typename Acc<MT>::T* yv;    // n_k  [s; psi]
  typename Acc<MT>::T* gv;    // n_v
  typename Acc<MT>::T* rv;    // n_v
  typename Acc<MT>::T* dv;    // n_v
  typename Acc<MT>::T* sv;    // n_x
  typename Acc<MT>::T* part;  // kThreads
  double* red;                // 3 * kWarps
  int* flag;                  // small ints
};

inline __host__ __device__ long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

// Padded sizes (entries) of the two matrices of a pack; multiples of 32 entries
// keep every bulk copy 16-byte aligned for all element types.
inline __host__ __device__ long long kpad(int n_k, int n_v) { return round_up((long long)n_k * n_v, 32); }
inline __host__ __device__ long long lpad(int n_v) { return round_up((long long)n_v * n_v, 32); }

template <typename MT>
__host__ __device__ size_t vec_smem_bytes(int n_x, int n_u, int n_v) {
  using AT = typename Acc<MT>::T;
  const int n_k = n_x + n_u;
  size_t v = (size_t)(n_k + 3 * n_v + n_x + kThreads) * sizeof(AT);
  v = round_up(v, 16);
  v += 3 * kWarps * sizeof(double) + 16 * sizeof(int);
  return round_up(v, 128);
}

template <typename MT>
__device__ Smem<MT> carve(unsigned char* base, int S, int n_x, int n_u, int n_v) {
  using AT = typename Acc<MT>::T;
  Smem<MT> s;
  const int n_k = n_x + n_u;
  size_t off = 0;
  for (int i = 0; i < S; ++i) {
    s.K[i] = reinterpret_cast<MT*>(base + off);
    off += kpad(n_k, n_v) * sizeof(MT);
  }
  for (int i = 0; i < S; ++i) {
    s.Lm[i] = reinterpret_cast<MT*>(base + off);
    off += lpad(n_v) * sizeof(MT);
  }
  off = round_up(off, 16);
  s.barK = reinterpret_cast<uint64_t*>(base + off);
  off += 4 * sizeof(uint64_t);
  s.barL = reinterpret_cast<uint64_t*>(base + off);
  off += 4 * sizeof(uint64_t);
  off = round_up(off, 16);
  AT* v = reinterpret_cast<AT*>(base + off);
  s.yv = v;
  v += n_k;
  s.gv = v;
  v += n_v;
  s.rv = v;
  v += n_v;
  s.dv = v;
  v += n_v;
  s.sv = v;
  v += n_x;
  s.part = v;
  v += kThreads;
  off = round_up(reinterpret_cast<unsigned char*>(v) - base, 16);
  s.red = reinterpret_cast<double*>(base + off);
  off += 3 * kWarps * sizeof(double);
  s.flag = reinterpret_cast<int*>(base + off);
  return s;
}

template <typename MT>
__host__ __device__ size_t iter_smem_bytes(int S, int n_x, int n_u, int n_v) {
  size_t m = (size_t)S * (kpad(n_x + n_u, n_v) + lpad(n_v)) * sizeof(MT);
  m = round_up(m, 16) + 8 * sizeof(uint64_t);
  m = round_up(m, 16);
  return m + vec_smem_bytes<MT>(n_x, n_u, n_v);
}

// Per-CTA cursor over the nodes of its chains, in backward (bottom-up) order.
struct Cursor {
  int chain;  // global chain index, or -1 when exhausted
  int k;      // position inside the chain (top-down index), counting down
};

struct Pipe {
  Cursor next_k, next_l;  // next node whose K / Lambda load is to be issued
  uint32_t issued_k, issued_l, used;
};

template <typename VT, typename MT>
struct Kern {
  using AT = typename Acc<MT>::T;
  const IterArgs& a;
  Smem<MT>& sm;
  int S, nu, mode;
  int nd;  // dual block 2 n_x + n_u

  __device__ Kern(const IterArgs& args, Smem<MT>& s, int S_, int nu_, int mode_)
      : a(args), sm(s), S(S_), nu(nu_), mode(mode_), nd(2 * args.n_x + args.n_u) {}

  __device__ VT* y(int k) const { return reinterpret_cast<VT*>((k & 1) ? a.ybuf1 : a.ybuf0); }
  __device__ VT* wb() const { return reinterpret_cast<VT*>(a.wbuf); }
  __device__ VT* hb() const { return reinterpret_cast<VT*>(a.h); }
  __device__ const VT* cv(const void* p) const { return reinterpret_cast<const VT*>(p); }
  __device__ VT* mv(void* p) const { return reinterpret_cast<VT*>(p); }
  __device__ const MT* pack(int n) const {
    return reinterpret_cast<const MT*>(a.packs) + (long long)n * a.pack_stride;
  }
  __device__ bool linear() const { return (mode & MODE_LINEAR) != 0; }

  // ---------------------------------------------------------- cursor helpers
  __device__ Cursor first_cursor() const {
    Cursor c;
    c.chain = blockIdx.x;
    if (c.chain >= a.n_chains) {
      c.chain = -1;
      c.k = 0;
      return c;
    }
    c.k = a.chain_off[c.chain + 1] - a.chain_off[c.chain] - 1;
    return c;
  }
  __device__ void advance(Cursor& c) const {
    if (c.chain < 0) return;
    if (--c.k < 0) {
      c.chain += gridDim.x;
      if (c.chain >= a.n_chains) {
        c.chain = -1;
        return;
      }
      c.k = a.chain_off[c.chain + 1] - a.chain_off[c.chain] - 1;
    }
  }
  __device__ int node_of(const Cursor& c) const { return a.chain_node[a.chain_off[c.chain] + c.k]; }

  // thread 0 only
  __device__ void issue_k(Pipe& p) {
    if (p.next_k.chain < 0) return;
    const int slot = p.issued_k % S;
    const int n = node_of(p.next_k);
    const uint32_t bytes = (uint32_t)(kpad(a.n_k, a.n_v) * sizeof(MT));
    mbar_expect_tx(&sm.barK[slot], bytes);
    const unsigned char* src = reinterpret_cast<const unsigned char*>(pack(n));
    unsigned char* dst = reinterpret_cast<unsigned char*>(sm.K[slot]);
    for (uint32_t o = 0; o < bytes; o += kChunk) bulk_g2s(dst + o, src + o, min((uint32_t)kChunk, bytes - o), &sm.barK[slot]);
    ++p.issued_k;
    advance(p.next_k);
  }
  __device__ void issue_l(Pipe& p) {
    if (p.next_l.chain < 0) return;
    const int slot = p.issued_l % S;
    const int n = node_of(p.next_l);
    const uint32_t bytes = (uint32_t)(lpad(a.n_v) * sizeof(MT));
    mbar_expect_tx(&sm.barL[slot], bytes);
    const unsigned char* src = reinterpret_cast<const unsigned char*>(pack(n) + kpad(a.n_k, a.n_v));
    unsigned char* dst = reinterpret_cast<unsigned char*>(sm.Lm[slot]);
    for (uint32_t o = 0; o < bytes; o += kChunk) bulk_g2s(dst + o, src + o, min((uint32_t)kChunk, bytes - o), &sm.barL[slot]);
    ++p.issued_l;
    advance(p.next_l);
  }

  // ---------------------------------------------------------- forward + prox
  // Path sums of the forward sweep for node `top` (inclusive) into thread-owned
  // accumulators: entry idx < n_x -> (V, X) of the states, else U of the inputs.
  __device__ void path_init(int node_or_neg, int idx, AT& V, AT& X, AT& U) const {
    V = 0;
    U = 0;
    X = (idx < a.n_x && !linear()) ? (AT)cv(a.p0)[idx] : (AT)0;
    if (node_or_neg < 0) return;
    const int b = a.path_off[node_or_neg], e = a.path_off[node_or_neg + 1];
    for (int q = b; q < e; ++q) step_forward(a.path_node[q], idx, V, X, U);
  }
  __device__ void step_forward(int m, int idx, AT& V, AT& X, AT& U) const {
    const VT* hm = hb() + (long long)m * a.n_k;
    if (idx < a.n_x) {
      V += (AT)hm[idx];
      X += V + (linear() ? (AT)0 : (AT)cv(a.e)[(long long)m * a.n_x + idx]);
    } else {
      U += (AT)hm[idx];
    }
  }
  __device__ void write_z(int m, int idx, AT X, AT U) const {
    if (idx < a.n_x)
      mv(a.xout)[(long long)m * a.n_x + idx] = (VT)X;
    else {
      const int i = idx - a.n_x;
      mv(a.uout)[(long long)m * a.n_u + i] =
          (VT)(U + (linear() ? (AT)0 : (AT)cv(a.uhat)[(long long)m * a.n_u + i]));
    }
  }

  // Prox, dual update and next extrapolation of node m by one warp.
  // Iteration it = nu - 1: reads y^{it} (buffer it) and y^{it-1} (buffer it+1),
  // writes y^{it+1} into buffer it+1 and w^{it+1} (xi, psi) into wbuf.
  __device__ void prox_node(int m, int lane, double& rmax, double& hzmax, double& tmax) {
    const int it = nu - 1;
    VT* y1 = y(it) + (long long)m * nd;
    VT* y2 = y(it + 1) + (long long)m * nd;
    const VT* xo = cv(a.xout) + (long long)m * a.n_x;
    const VT* uo = cv(a.uout) + (long long)m * a.n_u;
    VT* wm = wb() + (long long)m * a.n_k;
    if (linear()) {
      // power iteration: y_{k+1} = -D^{1/2} H z ; accumulate norms
      const AT ss = sqrt((AT)cv(a.step_s)[m]), sz = sqrt((AT)cv(a.step_z)[m]);
      double nrm = 0, dot = 0;
      for (int i = lane; i < a.n_x; i += 32) {
        const AT x = (AT)xo[i];
        const AT a1 = -ss * x, a2 = -sz * x;
        dot += (double)a1 * (double)y1[i] + (double)a2 * (double)y1[a.n_x + i];
        y2[i] = (VT)a1;
        y2[a.n_x + i] = (VT)a2;
        nrm += (double)a1 * a1 + (double)a2 * a2;
      }
      for (int i = lane; i < a.n_u; i += 32) {
        const AT u = (AT)uo[i];
        const AT a3 = -sqrt((AT)cv(a.step_p)[(long long)m * a.n_u + i]) * u;
        dot += (double)a3 * (double)y1[2 * a.n_x + i];
        y2[2 * a.n_x + i] = (VT)a3;
        nrm += (double)a3 * a3;
      }
      nrm = warp_sum(nrm);
      dot = warp_sum(dot);
      if (lane == 0) {
        atomicAdd(&a.pw[it + 1], nrm);
        atomicAdd(&a.pw[a.pw_len + it], dot);
      }
      return;
    }
    const AT c = (AT)a.cvec[it];
    const AT cn = (AT)a.cvec[it + 1];
    const AT ls = (AT)cv(a.step_s)[m], lz = (AT)cv(a.step_z)[m];
    const AT mu = (AT)cv(a.mu_s)[m];
    const VT* xs = cv(a.x_s);
    const VT* xlo = cv(a.x_min);
    const VT* xhi = cv(a.x_max);
    AT d2s = 0, d2z = 0;
    for (int i = lane; i < a.n_x; i += 32) {
      const AT x = (AT)xo[i];
      const AT ws = (AT)y1[i] + c * ((AT)y1[i] - (AT)y2[i]);
      const AT wz = (AT)y1[a.n_x + i] + c * ((AT)y1[a.n_x + i] - (AT)y2[a.n_x + i]);
      const AT vs = ws / ls + x, vz = wz / lz + x;
      const AT Ps = fmax(vs, (AT)xs[i]);
      const AT Pz = fmin(fmax(vz, (AT)xlo[i]), (AT)xhi[i]);
      d2s += (vs - Ps) * (vs - Ps);
      d2z += (vz - Pz) * (vz - Pz);
    }
    d2s = warp_sum(d2s);
    d2z = warp_sum(d2z);
    const AT ds = sqrt(d2s), dz = sqrt(d2z);
    const AT ths = mu / ls, thz = (AT)a.gamma_d / lz;
    const bool fs = ds > ths, fz = dz > thz;
    const AT ks = fs ? ths / ds : (AT)0, kz = fz ? thz / dz : (AT)0;
    bool bad = false;
    for (int i = lane; i < a.n_x; i += 32) {
      const AT x = (AT)xo[i];
      const AT y1s = (AT)y1[i], y1z = (AT)y1[a.n_x + i];
      const AT ws = y1s + c * (y1s - (AT)y2[i]);
      const AT wz = y1z + c * (y1z - (AT)y2[a.n_x + i]);
      const AT vs = ws / ls + x, vz = wz / lz + x;
      const AT Ps = fmax(vs, (AT)xs[i]);
      const AT Pz = fmin(fmax(vz, (AT)xlo[i]), (AT)xhi[i]);
      const AT ts = fs ? vs + ks * (Ps - vs) : Ps;
      const AT tz = fz ? vz + kz * (Pz - vz) : Pz;
      const AT ysn = ws + ls * (x - ts);
      const AT yzn = wz + lz * (x - tz);
      y2[i] = (VT)ysn;
      y2[a.n_x + i] = (VT)yzn;
      rmax = fmax(rmax, (double)fmax(fabs(x - ts), fabs(x - tz)));
      hzmax = fmax(hzmax, (double)fabs(x));
      tmax = fmax(tmax, (double)fmax(fabs(ts), fabs(tz)));
      const AT wsn = ysn + cn * (ysn - y1s);
      const AT wzn = yzn + cn * (yzn - y1z);
      wm[i] = (VT)(wsn + wzn);
      bad |= !isfinite(ysn) || !isfinite(yzn);
    }
    const VT* ulo = cv(a.u_min);
    const VT* uhi = cv(a.u_max);
    const VT* lp = cv(a.step_p) + (long long)m * a.n_u;
    for (int i = lane; i < a.n_u; i += 32) {
      const AT u = (AT)uo[i];
      const AT y1p = (AT)y1[2 * a.n_x + i];
      const AT wp = y1p + c * (y1p - (AT)y2[2 * a.n_x + i]);
      const AT l = (AT)lp[i];
      const AT vp = wp / l + u;
      const AT tp = fmin(fmax(vp, (AT)ulo[i]), (AT)uhi[i]);
      const AT ypn = wp + l * (u - tp);
      y2[2 * a.n_x + i] = (VT)ypn;
      rmax = fmax(rmax, (double)fabs(u - tp));
      hzmax = fmax(hzmax, (double)fabs(u));
      tmax = fmax(tmax, (double)fabs(tp));
      wm[a.n_x + i] = (VT)(ypn + cn * (ypn - y1p));
      bad |= !isfinite(ypn);
    }
    if (bad) a.flags[1] = SMPC_EDIVERGED;
  }

  // w^nu of node m without a prox (first iteration, or power iteration).
  __device__ void w_only_node(int m, int idx0, int stride) {
    VT* wm = wb() + (long long)m * a.n_k;
    if (linear()) {
      const double inv = rsqrt(a.pw[nu]);
      const VT* yk = y(nu) + (long long)m * nd;
      for (int idx = idx0; idx < a.n_k; idx += stride) {
        AT w;
        if (idx < a.n_x) {
          w = sqrt((AT)cv(a.step_s)[m]) * (AT)yk[idx] + sqrt((AT)cv(a.step_z)[m]) * (AT)yk[a.n_x + idx];
        } else {
          const int i = idx - a.n_x;
          w = sqrt((AT)cv(a.step_p)[(long long)m * a.n_u + i]) * (AT)yk[2 * a.n_x + i];
        }
        wm[idx] = (VT)(w * (AT)inv);
      }
      return;
    }
    const AT c = (AT)a.cvec[nu];
    const VT* ya = y(nu) + (long long)m * nd;
    const VT* yb = y(nu + 1) + (long long)m * nd;
    for (int idx = idx0; idx < a.n_k; idx += stride) {
      AT w;
      if (idx < a.n_x) {
        const AT s1 = (AT)ya[idx], z1 = (AT)ya[a.n_x + idx];
        w = (s1 + c * (s1 - (AT)yb[idx])) + (z1 + c * (z1 - (AT)yb[a.n_x + idx]));
      } else {
        const int i = idx - a.n_x;
        const AT p1 = (AT)ya[2 * a.n_x + i];
        w = p1 + c * (p1 - (AT)yb[2 * a.n_x + i]);
      }
      wm[idx] = (VT)w;
    }
  }

  // ---------------------------------------------------------- backward pieces
  // r := r + [Bbar; L]' yv (K in A), publish, delta = Lam r, h = K delta.
  __device__ void node_tail(int m, const MT* K, const MT* Lam) {
    matvec_t<MT, AT>(K, a.n_k, a.n_v, sm.yv, sm.gv, sm.part);
    for (int j = threadIdx.x; j < a.n_v; j += kThreads) sm.rv[j] += sm.gv[j];
    __syncthreads();
    matvec_t<MT, AT>(Lam, a.n_v, a.n_v, sm.rv, sm.dv, sm.part);  // Lambda symmetric
  }

  // Process top node t with the whole CTA (its children are complete).
  __device__ void process_top(int t) {
    const MT* K = pack(t);
    const MT* Lam = K + kpad(a.n_k, a.n_v);
    const int cb = a.child_begin[t], cc = a.child_count[t];
    const VT* wt = wb() + (long long)t * a.n_k;
    for (int idx = threadIdx.x; idx < a.n_k; idx += kThreads) {
      AT v = (AT)ldcg(wt + idx);
      if (idx < a.n_x) {
        for (int c = cb; c < cb + cc; ++c) v += (AT)ldcg(mv(a.spub) + (long long)c * a.n_x + idx);
        sm.sv[idx] = v;
      }
      sm.yv[idx] = v;
    }
    for (int j = threadIdx.x; j < a.n_v; j += kThreads) {
      AT r = linear() ? (AT)0 : (AT)cv(a.beta)[(long long)t * a.n_v + j];
      for (int c = cb; c < cb + cc; ++c) r += (AT)ldcg(mv(a.rpub) + (long long)c * a.n_v + j);
      sm.rv[j] = r;
    }
    __syncthreads();
    node_tail(t, K, Lam);
    for (int i = threadIdx.x; i < a.n_x; i += kThreads) mv(a.spub)[(long long)t * a.n_x + i] = (VT)sm.sv[i];
    for (int j = threadIdx.x; j < a.n_v; j += kThreads) mv(a.rpub)[(long long)t * a.n_v + j] = (VT)sm.rv[j];
    matvec_n<MT, AT>(K, a.n_k, a.n_v, sm.dv, sm.yv, sm.part);
    for (int i = threadIdx.x; i < a.n_k; i += kThreads) hb()[(long long)t * a.n_k + i] = (VT)sm.yv[i];
    __syncthreads();
  }

  // Arrive at top node t; while this CTA is the last arrival, process and climb.
  __device__ void arrive_and_climb(int t) {
    while (t >= 0) {
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        const int old = atomicAdd(&a.counters[t], 1);
        const int last = (old == a.top_expect[t] - 1);
        if (last) {
          a.counters[t] = 0;  // nobody else touches it again in this launch
          __threadfence();
        }
        sm.flag[0] = last;
      }
      __syncthreads();
      if (!sm.flag[0]) return;
      process_top(t);
      t = a.parent[t];
    }
  }

  // A bounded wait gave up: flag the error, let this CTA's copies in flight land
  // (again with a bound) so no bulk copy outlives the CTA's shared memory, return.
  __device__ void drain(const Pipe& p) {
    if (threadIdx.x == 0) a.flags[1] = SMPC_ETIMEOUT;
    for (uint32_t q = p.used; q < p.issued_k; ++q) mbar_wait(&sm.barK[q % S], (q / S) & 1);
    for (uint32_t q = p.used; q < p.issued_l; ++q) mbar_wait(&sm.barL[q % S], (q / S) & 1);
    __syncthreads();
  }

  // ---------------------------------------------------------- the launch
  __device__ void run() {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double rmax = 0, hzmax = 0, tmax = 0;
    const bool do_prox = (mode & MODE_PROX) != 0 && nu >= 1;
    const bool do_bwd = (mode & MODE_BWD) != 0;

    // pipeline set-up
    Pipe p;
    p.next_k = p.next_l = first_cursor();
    p.issued_k = p.issued_l = p.used = 0;
    if (tid == 0) {
      for (int s = 0; s < S; ++s) {
        mbar_init(&sm.barK[s], 1);
        mbar_init(&sm.barL[s], 1);
      }
      fence_barrier_init();
      fence_proxy_async();
    }
    __syncthreads();
    if (do_bwd && tid == 0) {
      for (int s = 0; s < S; ++s) {
        issue_k(p);
        issue_l(p);
      }
    }

    // top-node tasks: forward + prox (Phase P), then w^nu and the arrival
    for (int ti = blockIdx.x; ti < a.n_top; ti += gridDim.x) {
      const int t = a.top_nodes[ti];
      if (do_prox) {
        for (int idx = tid; idx < a.n_k; idx += kThreads) {
          AT V, X, U;
          path_init(t, idx, V, X, U);
          write_z(t, idx, X, U);
        }
        __syncthreads();
        if (warp == 0) prox_node(t, lane, rmax, hzmax, tmax);
        __syncthreads();
      }
      if (do_bwd) {
        if (!do_prox || linear()) w_only_node(t, tid, kThreads);
        arrive_and_climb(t);
      }
    }

    // chains
    for (int ch = blockIdx.x; ch < a.n_chains; ch += gridDim.x) {
      const int cb = a.chain_off[ch], len = a.chain_off[ch + 1] - cb;
      const int* nodes = a.chain_node + cb;
      if (do_prox) {
        const int par = a.chain_parent[ch];
        for (int idx = tid; idx < a.n_k; idx += kThreads) {
          AT V, X, U;
          path_init(par, idx, V, X, U);
          for (int k = 0; k < len; ++k) {
            step_forward(nodes[k], idx, V, X, U);
            write_z(nodes[k], idx, X, U);
          }
        }
        __syncthreads();
        for (int k = warp; k < len; k += kWarps) prox_node(nodes[k], lane, rmax, hzmax, tmax);
        __syncthreads();
      }
      if (!do_bwd) continue;
      if (!do_prox || linear()) {
        for (int k = 0; k < len; ++k) w_only_node(nodes[k], tid, kThreads);
        __syncthreads();
      }
      // backward along the chain, bottom-up
      for (int i = tid; i < a.n_x; i += kThreads) sm.sv[i] = 0;
      for (int j = tid; j < a.n_v; j += kThreads) sm.rv[j] = 0;
      __syncthreads();
      for (int k = len - 1; k >= 0; --k) {
        const int m = nodes[k];
        const VT* wm = wb() + (long long)m * a.n_k;
        for (int idx = tid; idx < a.n_k; idx += kThreads) {
          AT v = (AT)wm[idx];
          if (idx < a.n_x) {
            v += sm.sv[idx];
            sm.sv[idx] = v;
          }
          sm.yv[idx] = v;
        }
        if (!linear())
          for (int j = tid; j < a.n_v; j += kThreads) sm.rv[j] += (AT)cv(a.beta)[(long long)m * a.n_v + j];
        const int slot = p.used % S;
        const uint32_t par = (p.used / S) & 1;
        if (__syncthreads_or(!mbar_wait(&sm.barK[slot], par))) {
          drain(p);
          return;
        }
        matvec_t<MT, AT>(sm.K[slot], a.n_k, a.n_v, sm.yv, sm.gv, sm.part);
        for (int j = tid; j < a.n_v; j += kThreads) sm.rv[j] += sm.gv[j];
        if (__syncthreads_or(!mbar_wait(&sm.barL[slot], par))) {
          drain(p);
          return;
        }
        matvec_t<MT, AT>(sm.Lm[slot], a.n_v, a.n_v, sm.rv, sm.dv, sm.part);
        if (tid == 0) {  // Lambda slot is free: refill it
          fence_proxy_async();
          issue_l(p);
        }
        matvec_n<MT, AT>(sm.K[slot], a.n_k, a.n_v, sm.dv, sm.yv, sm.part);
        VT* hm = hb() + (long long)m * a.n_k;
        for (int i = tid; i < a.n_k; i += kThreads) hm[i] = (VT)sm.yv[i];
        if (tid == 0) {  // K slot is free (matvec_n ended with a barrier)
          fence_proxy_async();
          issue_k(p);
        }
        ++p.used;
        __syncthreads();  // yv is rewritten by the next node
      }
      // publish the chain head's s and r, arrive at its top parent
      const int head = nodes[0];
      for (int i = tid; i < a.n_x; i += kThreads) mv(a.spub)[(long long)head * a.n_x + i] = (VT)sm.sv[i];
      for (int j = tid; j < a.n_v; j += kThreads) mv(a.rpub)[(long long)head * a.n_v + j] = (VT)sm.rv[j];
      arrive_and_climb(a.chain_parent[ch]);
    }

    if (do_prox && !linear()) {  // residual of iteration nu - 1 (Sec. IV-E)
      rmax = warp_max(rmax);
      hzmax = warp_max(hzmax);
      tmax = warp_max(tmax);
      if (lane == 0) {
        sm.red[warp] = rmax;
        sm.red[kWarps + warp] = hzmax;
        sm.red[2 * kWarps + warp] = tmax;
      }
      __syncthreads();
      if (tid == 0) {
        double r = 0, hz = 0, tt = 0;
        for (int w = 0; w < kWarps; ++w) {
          r = fmax(r, sm.red[w]);
          hz = fmax(hz, sm.red[kWarps + w]);
          tt = fmax(tt, sm.red[2 * kWarps + w]);
        }
        unsigned long long* slot = a.res + 3ll * (nu - 1);
        atomic_max_nonneg(slot + 0, r);
        atomic_max_nonneg(slot + 1, hz);
        atomic_max_nonneg(slot + 2, tt);
      }
    }
  }
};

template <typename VT, typename MT>
__global__ void __launch_bounds__(kThreads, 1)
    apg_iter(const __grid_constant__ IterArgs a, int S, int nu, int mode) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Smem<MT> sm = carve<MT>(smem_raw, S, a.n_x, a.n_u, a.n_v);
  // uniform early exit: stopped, failed, or converged two iterations ago
  if (threadIdx.x == 0) {
    int stop = 0;
    if (mode & MODE_CHECK) {
      const int done = ldcg(a.flags + 0), err = ldcg(a.flags + 1);
      if (done >= 0 || err != 0) stop = 1;
      if (!stop && a.tol > 0 && nu >= 2) {
        const unsigned long long* r = a.res + 3ll * (nu - 2);
        const double rho = __longlong_as_double((long long)ldcg(r + 0));
        const double hz = __longlong_as_double((long long)ldcg(r + 1));
        const double tt = __longlong_as_double((long long)ldcg(r + 2));
        if (rho / (1.0 + fmax(hz, tt)) <= a.tol) {
          stop = 1;
          if (blockIdx.x == 0) a.flags[0] = nu - 1;
        }
      }
    }
    sm.flag[1] = stop;
  }
  __syncthreads();
  if (sm.flag[1]) return;
  Kern<VT, MT> k(a, sm, S, nu, mode);
  k.run();
}

// ------------------------------------------------------------------ helpers
template <typename VT, typename MT>
__global__ void pack_kernel(int n, int n_k, int n_v, const double* K, const double* Lam, const double* prob,
                            MT* packs, long long stride) {
  const long long kp = kpad(n_k, n_v), lp = lpad(n_v);
  for (int m = blockIdx.x; m < n; m += gridDim.x) {
    MT* dst = packs + (long long)m * stride;
    const double inv = 1.0 / (2.0 * prob[m]);
    for (long long i = threadIdx.x; i < kp; i += blockDim.x)
      dst[i] = (MT)(i < (long long)n_k * n_v ? K[i] : 0.0);
    for (long long i = threadIdx.x; i < lp; i += blockDim.x)
      dst[kp + i] = (MT)(i < (long long)n_v * n_v ? Lam[i] * inv : 0.0);
  }
}

template <typename VT>
__global__ void cost_alpha_kernel(CostArgs a) {
  // alpha_bar_j = L' W_alpha (alpha_1 + alpha_{2,j})
  for (int j = blockIdx.x; j < a.N; j += gridDim.x)
    for (int k = threadIdx.x; k < a.n_v; k += blockDim.x) {
      double s = 0;
      for (int i = 0; i < a.n_u; ++i) s += a.L[(long long)i * a.n_v + k] * a.W_alpha * (a.alpha1[i] + a.alpha2[(long long)j * a.n_u + i]);
      a.abar[(long long)j * a.n_v + k] = s;
    }
}

template <typename VT>
__global__ void cost_uhat_kernel(CostArgs a) {
  // d_n = dhat_j + eps_n ; u_hat_n = Pu d_n ; e_n = Pe d_n
  extern __shared__ double dsh[];
  for (int m = blockIdx.x; m < a.n; m += gridDim.x) {
    const int j = a.stage[m];
    for (int i = threadIdx.x; i < a.n_d; i += blockDim.x)
      dsh[i] = a.dhat[(long long)j * a.n_d + i] + a.eps[(long long)m * a.n_d + i];
    __syncthreads();
    for (int i = threadIdx.x; i < a.n_u + a.n_x; i += blockDim.x) {
      const double* row = (i < a.n_u) ? a.Pu + (long long)i * a.n_d : a.Pe + (long long)(i - a.n_u) * a.n_d;
      double s = 0;
      for (int k = 0; k < a.n_d; ++k) s += row[k] * dsh[k];
      if (i < a.n_u) {
        a.uhat64[(long long)m * a.n_u + i] = s;
        reinterpret_cast<VT*>(a.uhat)[(long long)m * a.n_u + i] = (VT)s;
      } else {
        reinterpret_cast<VT*>(a.e)[(long long)m * a.n_x + (i - a.n_u)] = (VT)s;
      }
    }
    __syncthreads();
  }
}

template <typename VT>
__global__ void cost_beta_kernel(CostArgs a) {
  // beta_n = p_n abar_j + 2 Rhat' (pbar_n u_hat_n - p_n u_hat_pi - sum_c p_c u_hat_c), u_hat_pi(root) = q
  extern __shared__ double Dsh[];
  for (int m = blockIdx.x; m < a.n; m += gridDim.x) {
    const double pm = a.prob[m];
    const int par = a.parent[m];
    const int cb = a.child_begin[m], cc = a.child_count[m];
    for (int i = threadIdx.x; i < a.n_u; i += blockDim.x) {
      double D = a.pbar[m] * a.uhat64[(long long)m * a.n_u + i];
      D -= pm * (par >= 0 ? a.uhat64[(long long)par * a.n_u + i] : a.q[i]);
      for (int c = cb; c < cb + cc; ++c) D -= a.prob[c] * a.uhat64[(long long)c * a.n_u + i];
      Dsh[i] = D;
    }
    __syncthreads();
    const int j = a.stage[m];
    for (int k = threadIdx.x; k < a.n_v; k += blockDim.x) {
      double s = 0;
      for (int i = 0; i < a.n_u; ++i) s += a.Rhat[(long long)i * a.n_v + k] * Dsh[i];
      reinterpret_cast<VT*>(a.beta)[(long long)m * a.n_v + k] = (VT)(pm * a.abar[(long long)j * a.n_v + k] + 2.0 * s);
    }
    __syncthreads();
  }
}

template <typename VT>
__global__ void final_y_kernel(IterArgs a, int max_iters, VT* dst) {
  __shared__ int it;
  if (threadIdx.x == 0) {
    it = a.flags[0];
    if (it < 0) it = max_iters;
  }
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0) a.flags[0] = it;
  if (!dst) return;
  const VT* src = reinterpret_cast<const VT*>((it & 1) ? a.ybuf1 : a.ybuf0);
  const long long total = (long long)a.n * (2 * a.n_x + a.n_u);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

template <typename VT>
__global__ void init_duals_kernel(IterArgs a, int warm) {
  // cold: y^0 = y^{-1} = 0 ; warm: both = the final dual of the previous solve
  const long long total = (long long)a.n * (2 * a.n_x + a.n_u);
  int it = a.flags[0];
  const VT* src = reinterpret_cast<const VT*>((it & 1) ? a.ybuf1 : a.ybuf0);
  VT* y0 = reinterpret_cast<VT*>(a.ybuf0);
  VT* y1 = reinterpret_cast<VT*>(a.ybuf1);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const VT v = warm ? src[i] : (VT)0;
    y0[i] = v;
    y1[i] = v;
  }
}

template <typename VT>
__global__ void convert_kernel(const double* src, VT* dst, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (VT)src[i];
}

int check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return SMPC_ECUDA;
  }
  return SMPC_OK;
}

template <typename VT, typename MT>
LaunchCfg config_t(const IterArgs& a, int num_sms, int S_max) {
  LaunchCfg c;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (optin <= 0) optin = 232448;
  int S = S_max;
  while (S > 1 && iter_smem_bytes<MT>(S, a.n_x, a.n_u, a.n_v) > (size_t)optin) --S;
  c.stages = S;
  c.smem = iter_smem_bytes<MT>(S, a.n_x, a.n_u, a.n_v);
  if (c.smem > (size_t)optin) c.stages = 0;
  c.block = kThreads;
  c.grid = a.n_chains < num_sms ? a.n_chains : num_sms;
  if (c.grid < 1) c.grid = 1;
  return c;
}

template <typename VT, typename MT>
int launch_t(const IterArgs& a, const LaunchCfg& c, int nu, int mode, cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(apg_iter<VT, MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    attr_set = true;
  }
  apg_iter<VT, MT><<<c.grid, c.block, c.smem, s>>>(a, c.stages, nu, mode);
  return check_launch("apg_iter");
}

}  // namespace

size_t vec_size(int prec) { return prec == SMPC_FP64 ? sizeof(double) : sizeof(float); }
size_t mat_size(int prec) {
  return prec == SMPC_FP64 ? sizeof(double) : prec == SMPC_FP32 ? sizeof(float) : sizeof(__nv_bfloat16);
}
long long pack_entries(int n_k, int n_v) { return kpad(n_k, n_v) + lpad(n_v); }

LaunchCfg iter_config(int prec, const IterArgs& a, int num_sms) {
  switch (prec) {
    case SMPC_FP64: return config_t<double, double>(a, num_sms, 1);
    case SMPC_FP32: return config_t<float, float>(a, num_sms, 2);
    default: return config_t<float, __nv_bfloat16>(a, num_sms, 4);
  }
}

int launch_iter(int prec, const IterArgs& a, const LaunchCfg& c, int nu, int mode, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (prec) {
    case SMPC_FP64: return launch_t<double, double>(a, c, nu, mode, s);
    case SMPC_FP32: return launch_t<float, float>(a, c, nu, mode, s);
    default: return launch_t<float, __nv_bfloat16>(a, c, nu, mode, s);
  }
}

int launch_pack(int prec, int n, int n_k, int n_v, const double* K, const double* Lam, const double* prob,
                void* packs, long long stride, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int grid = n < 4096 ? n : 4096;
  switch (prec) {
    case SMPC_FP64:
      pack_kernel<double, double><<<grid, 256, 0, s>>>(n, n_k, n_v, K, Lam, prob, (double*)packs, stride);
      break;
    case SMPC_FP32:
      pack_kernel<float, float><<<grid, 256, 0, s>>>(n, n_k, n_v, K, Lam, prob, (float*)packs, stride);
      break;
    default:
      pack_kernel<float, __nv_bfloat16><<<grid, 256, 0, s>>>(n, n_k, n_v, K, Lam, prob, (__nv_bfloat16*)packs, stride);
  }
  return check_launch("pack_kernel");
}

int launch_cost_update(int prec, const CostArgs& a, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int grid = a.n < 4096 ? a.n : 4096;
  const size_t sh1 = (size_t)a.n_d * sizeof(double), sh2 = (size_t)a.n_u * sizeof(double);
  if (prec == SMPC_FP64) {
    cost_alpha_kernel<double><<<a.N, 128, 0, s>>>(a);
    cost_uhat_kernel<double><<<grid, 128, sh1, s>>>(a);
    cost_beta_kernel<double><<<grid, 128, sh2, s>>>(a);
  } else {
    cost_alpha_kernel<float><<<a.N, 128, 0, s>>>(a);
    cost_uhat_kernel<float><<<grid, 128, sh1, s>>>(a);
    cost_beta_kernel<float><<<grid, 128, sh2, s>>>(a);
  }
  return check_launch("cost_update");
}

int launch_copy_final_y(int prec, const IterArgs& a, int max_iters, void* dst, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (prec == SMPC_FP64)
    final_y_kernel<double><<<dst ? 256 : 1, 256, 0, s>>>(a, max_iters, (double*)dst);
  else
    final_y_kernel<float><<<dst ? 256 : 1, 256, 0, s>>>(a, max_iters, (float*)dst);
  return check_launch("final_y");
}

int launch_init_duals(int prec, const IterArgs& a, int warm, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (prec == SMPC_FP64)
    init_duals_kernel<double><<<256, 256, 0, s>>>(a, warm);
  else
    init_duals_kernel<float><<<256, 256, 0, s>>>(a, warm);
  return check_launch("init_duals");
}

int launch_convert(int prec, const double* src, void* dst, long long count, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (count <= 0) return SMPC_OK;
  const int grid = (int)((count + 255) / 256 < 1024 ? (count + 255) / 256 : 1024);
  if (prec == SMPC_FP64)
    convert_kernel<double><<<grid, 256, 0, s>>>(src, (double*)dst, count);
  else
    convert_kernel<float><<<grid, 256, 0, s>>>(src, (float*)dst, count);
  return check_launch("convert");
}

}  // namespace smpc
