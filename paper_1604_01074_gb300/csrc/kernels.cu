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
#include <type_traits>

#include "smpc_internal.h"

namespace smpc {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
// One bulk copy per matrix: on this GPU the copies one SM issues are served one
// after the other at a roughly fixed cost each, so per-SM bandwidth grows with the
// copy size (16 KB copies: ~54 GB/s per SM; 64 KB and larger: ~200 GB/s).
constexpr int kChunk = 1 << 20;          // larger than any matrix of a pack
constexpr uint64_t kWaitNs = 2000000000ull;  // bounded mbarrier wait: 2 s
constexpr int kMaxSlots = 4;                 // pack slots per CTA: one mbarrier each (barK, barL)

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
// One 4- or 8-byte element copied into shared memory by cp.async: the copies of a
// thread are issued back to back without holding registers and complete at
// cp_async_wait_all, after which the issuing thread sees them (others after a barrier).
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(dst)),
               "l"((unsigned long long)__cvta_generic_to_global(src)), "n"((int)sizeof(T))
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// Programmatic dependent launch: the iteration kernels let the next kernel of the
// stream be scheduled as soon as they start (its CTAs take free SM slots while this
// grid drains), and each waits for the previous grid to complete, with its memory
// visible, before it touches anything.  Without the launch attribute both are no-ops.
__device__ __forceinline__ void grid_dep_sync() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
// Release / acquire fence at GPU scope for the arrival counters: after a block barrier,
// thread 0's fence makes the whole CTA's prior writes visible before its arrival (the
// fence is cumulative over what the barrier ordered before it), and the last arriver's
// fence orders its reads of the other CTAs' results after their arrivals.
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
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
// Non-blocking test of phase `parity` of barrier b.
__device__ __forceinline__ bool mbar_test_now(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for phase `parity` of barrier b; gives up after limit_ns and returns false
// (limit 0: one non-blocking test).  Waits that let copies already in flight land
// before a CTA leaves always take the long bound kWaitNs.
__device__ bool mbar_wait(uint64_t* b, uint32_t parity, uint64_t limit_ns = kWaitNs) {
  if (limit_ns == 0) return mbar_test_now(b, parity);
  if (mbar_test(b, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_test(b, parity)) {
    if (global_ns() - t0 > limit_ns) return false;
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

// Forests with a stop per tree: tree r takes no further forward-sweep or prox writes from
// launch nu on once it stopped, i.e. when its own relative residual of iteration nu - 2 (or
// an earlier one) met tol.  Every kernel reaches the same answer: the residual of nu - 2 is
// final when launch nu starts, and tree_done records earlier stops.
__device__ __forceinline__ bool tree_stops(const unsigned long long* q, double tol) {
  const double rho = __longlong_as_double((long long)ldcg(q + 0));
  const double hz = __longlong_as_double((long long)ldcg(q + 1));
  const double tt = __longlong_as_double((long long)ldcg(q + 2));
  return rho / (1.0 + fmax(hz, tt)) <= tol;
}
__device__ __forceinline__ bool tree_active(const IterArgs& a, int r, int nu) {
  if (!a.res_tree) return true;
  if (ldcg(a.tree_done + r) >= 0) return false;
  if (!(a.tol > 0) || nu < 2) return true;
  return !tree_stops(a.res_tree + 3ll * ((long long)(nu - 2) * a.R + r), a.tol);
}
// per-tree residual maxima of a CTA, combined in shared memory when the forest is small
constexpr int kTreeTable = 64;
__device__ __forceinline__ void tree_res_add(const IterArgs& a, unsigned long long* table, int r, int nu, double rm,
                                             double hm, double tm) {
  if (a.R <= kTreeTable) {
    atomic_max_nonneg(table + 3 * r + 0, rm);
    atomic_max_nonneg(table + 3 * r + 1, hm);
    atomic_max_nonneg(table + 3 * r + 2, tm);
  } else {
    unsigned long long* q = a.res_tree + 3ll * ((long long)(nu - 1) * a.R + r);
    atomic_max_nonneg(q + 0, rm);
    atomic_max_nonneg(q + 1, hm);
    atomic_max_nonneg(q + 2, tm);
  }
}
__device__ __forceinline__ void tree_table_clear(const IterArgs& a, unsigned long long* table) {
  if (a.res_tree && a.R <= kTreeTable)
    for (int q = threadIdx.x; q < 3 * a.R; q += blockDim.x) table[q] = 0;
}
// after a block barrier: the CTA's table into the iteration's per-tree residuals
__device__ __forceinline__ void tree_table_flush(const IterArgs& a, const unsigned long long* table, int nu) {
  if (!a.res_tree || a.R > kTreeTable) return;
  unsigned long long* dst = a.res_tree + 3ll * (long long)(nu - 1) * a.R;
  for (int q = threadIdx.x; q < 3 * a.R; q += blockDim.x)
    if (table[q]) atomicMax(dst + q, table[q]);
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
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ------------------------------------------------------------------ dual state
// Late in a solve the dual iterates move by lambda (H z - t) per iteration, far
// below the rounding unit of |y| in float32: a float32 dual state rounds those
// moves away and the iteration stalls well above a useful residual.  Factors with
// float32 or bfloat16 packs therefore hold y^nu and y^{nu-1} as unevaluated sums
// hi + lo of two float32 (about 48 significant bits) and update them with
// error-free transformations built from float32 operations: TwoSum (Knuth, TAOCP
// vol. 2, Sec. 4.2.2), FastTwoSum and the product error through a fused
// multiply-add (Dekker, 1971).  float64 factors hold the state in float64.  Both
// take 8 bytes per entry.  The solve step itself reads w rounded to its vector type.
struct DS {
  float hi, lo;
};
template <typename VT>
struct St;
template <>
struct St<double> { using T = double; };
template <>
struct St<float> { using T = DS; };

// exact sum a + b = s + e, valid when |a| >= |b| or a = 0
__device__ __forceinline__ DS fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
// exact sum a + b = s + e for any a, b
__device__ __forceinline__ DS two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ DS st_add(DS x, DS y) {
  const DS t = two_sum(x.hi, y.hi);
  return fast_two_sum(t.hi, __fadd_rn(t.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ DS st_sub(DS x, DS y) { return st_add(x, DS{-y.hi, -y.lo}); }
// k x
__device__ __forceinline__ DS st_scale(DS x, float k) {
  const float p = __fmul_rn(x.hi, k);
  const float e = __fmaf_rn(x.lo, k, __fmaf_rn(x.hi, k, -p));
  return fast_two_sum(p, e);
}
// w + l d with the product l d taken exactly
__device__ __forceinline__ DS st_axpy(DS w, float l, float d) {
  const float p = __fmul_rn(l, d);
  const float pe = __fmaf_rn(l, d, -p);
  const DS t = two_sum(w.hi, p);
  return fast_two_sum(t.hi, __fadd_rn(t.lo, __fadd_rn(w.lo, pe)));
}
__device__ __forceinline__ float st_val(DS x) { return __fadd_rn(x.hi, x.lo); }
__device__ __forceinline__ bool st_pos(DS x) { return x.hi > 0.f; }
__device__ __forceinline__ bool st_neg(DS x) { return x.hi < 0.f; }
template <typename ST>
__device__ __forceinline__ ST st_from(double v);
template <>
__device__ __forceinline__ DS st_from<DS>(double v) { return DS{(float)v, 0.f}; }

__device__ __forceinline__ double st_add(double x, double y) { return x + y; }
__device__ __forceinline__ double st_sub(double x, double y) { return x - y; }
__device__ __forceinline__ double st_scale(double x, double k) { return x * k; }
__device__ __forceinline__ double st_axpy(double w, double l, double d) { return fma(l, d, w); }
__device__ __forceinline__ double st_val(double x) { return x; }
__device__ __forceinline__ bool st_pos(double x) { return x > 0.0; }
__device__ __forceinline__ bool st_neg(double x) { return x < 0.0; }
template <>
__device__ __forceinline__ double st_from<double>(double v) { return v; }

// extrapolation y1 + c (y1 - y2) of eq. optim:acceleration
template <typename ST, typename AT>
__device__ __forceinline__ ST st_extrap(ST y1, ST y2, AT c) {
  return st_add(y1, st_scale(st_sub(y1, y2), c));
}
// The same extrapolation rounded to the vector type, for a w that is stored in it: the
// difference of the two states and the product in single operations, within about one
// unit in the last place of the float result (float64 state: exact up to rounding).
__device__ __forceinline__ float st_extrap_val(DS y1, DS y2, float c) {
  const float d = __fadd_rn(__fsub_rn(y1.hi, y2.hi), __fsub_rn(y1.lo, y2.lo));
  return __fadd_rn(y1.hi, __fmaf_rn(c, d, y1.lo));
}
__device__ __forceinline__ double st_extrap_val(double y1, double y2, double c) { return fma(c, y1 - y2, y1); }
// lambda r of a box block (App. C): with q_hi = w + lambda (x - hi) and
// q_lo = w + lambda (x - lo) (q_hi <= q_lo), lambda r = q_hi where q_hi > 0,
// q_lo where q_lo < 0, and 0 inside the box.
template <typename ST>
__device__ __forceinline__ ST box_lr(ST qh, ST ql) {
  return st_pos(qh) ? qh : (st_neg(ql) ? ql : st_from<ST>(0.0));
}

// ------------------------------------------------------------------ CTA mat-vecs
// Matrices sit in shared memory row-major with a row stride `ld` (entries) that is
// a multiple of 16 bytes, so every access below is a 128-bit shared-memory load:
// 4 float32, 2 float64 or 8 bfloat16 matrix entries per instruction.
template <typename MT>
struct Vec;
template <>
struct Vec<float> { static constexpr int V = 4; };
template <>
struct Vec<double> { static constexpr int V = 2; };
template <>
struct Vec<__nv_bfloat16> { static constexpr int V = 8; };

template <typename MT>
inline __host__ __device__ int row_stride(int n_v) {
  const int V = 16 / (int)sizeof(MT);
  return (n_v + V - 1) / V * V;
}

__device__ __forceinline__ void ld16(const float* p, float (&o)[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
}
__device__ __forceinline__ void ld16(const double* p, double (&o)[2]) {
  const double2 t = *reinterpret_cast<const double2*>(p);
  o[0] = t.x; o[1] = t.y;
}
// bfloat16 -> float32 is a 16-bit shift of the bit pattern
__device__ __forceinline__ void ld16(const __nv_bfloat16* p, float (&o)[8]) {
  const uint4 t = *reinterpret_cast<const uint4*>(p);
  o[0] = __uint_as_float(t.x << 16); o[1] = __uint_as_float(t.x & 0xffff0000u);
  o[2] = __uint_as_float(t.y << 16); o[3] = __uint_as_float(t.y & 0xffff0000u);
  o[4] = __uint_as_float(t.z << 16); o[5] = __uint_as_float(t.z & 0xffff0000u);
  o[6] = __uint_as_float(t.w << 16); o[7] = __uint_as_float(t.w & 0xffff0000u);
}
// V accumulation-type entries of a 16-byte aligned vector
__device__ __forceinline__ void ldx(const float* p, float (&o)[4]) { ld16(p, o); }
__device__ __forceinline__ void ldx(const double* p, double (&o)[2]) { ld16(p, o); }
__device__ __forceinline__ void ldx(const float* p, float (&o)[8]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  const float4 b = *reinterpret_cast<const float4*>(p + 4);
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
}
// V accumulation-type entries to a 16-byte aligned vector (one or two vector stores)
__device__ __forceinline__ void st16(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st16(double* p, const double (&v)[2]) {
  *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
}
__device__ __forceinline__ void st16(float* p, const float (&v)[8]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  *reinterpret_cast<float4*>(p + 4) = make_float4(v[4], v[5], v[6], v[7]);
}

// out[j] = sum_i A[i*ld + j] x[i] for j < C (A' x), A with R rows.  Thread
// (g, p) accumulates columns g*V .. g*V+V-1 over the p-th slice of the rows; the
// slices are then added in a fixed order (deterministic).
template <typename MT, typename AT>
__device__ void matvec_t(const MT* A, int R, int C, int ld, const AT* x, AT* out, AT* part) {
  constexpr int V = Vec<MT>::V;
  const int t = threadIdx.x;
  const int G = ld / V;
  int P = kThreads / G;
  if (P > 16) P = 16;
  const int rc = (R + P - 1) / P;
  if (t < P * G) {
    const int g = t % G, p = t / G;
    const int i0 = p * rc, i1 = min(R, i0 + rc);
    AT acc[V];
#pragma unroll
    for (int k = 0; k < V; ++k) acc[k] = 0;
    const MT* col = A + g * V;
#pragma unroll 4
    for (int i = i0; i < i1; ++i) {
      AT av[V];
      ld16(col + (long long)i * ld, av);
      const AT xi = x[i];
#pragma unroll
      for (int k = 0; k < V; ++k) acc[k] += av[k] * xi;
    }
    AT* dst = part + p * ld + g * V;
#pragma unroll
    for (int k = 0; k < V; ++k) dst[k] = acc[k];
  }
  __syncthreads();
  for (int j = t; j < C; j += kThreads) {
    AT v[16];
#pragma unroll
    for (int p = 0; p < 16; ++p) v[p] = p < P ? part[p * ld + j] : (AT)0;  // independent loads
    AT s = 0;
#pragma unroll
    for (int p = 0; p < 16; ++p) s += v[p];  // fixed order: deterministic
    out[j] = s;
  }
  __syncthreads();
}

// out[i] = sum_j A[i*ld + j] x[j] for i < R (A x); x is 16-byte aligned with ld
// entries, zero beyond the true width.
template <typename MT, typename AT>
__device__ void matvec_n(const MT* A, int R, int ld, const AT* x, AT* out) {
  constexpr int V = Vec<MT>::V;
  const int G = ld / V;
  for (int i = threadIdx.x; i < R; i += kThreads) {
    const MT* row = A + (long long)i * ld;
    AT acc0 = 0, acc1 = 0;
#pragma unroll 4
    for (int g = 0; g < G; ++g) {
      AT av[V], xv[V];
      ld16(row + g * V, av);
      ldx(x + g * V, xv);
#pragma unroll
      for (int k = 0; k < V; k += 2) {
        acc0 += av[k] * xv[k];
        acc1 += av[k + 1] * xv[k + 1];
      }
    }
    out[i] = acc0 + acc1;
  }
  __syncthreads();
}

// ------------------------------------------------------------------ kernel state
constexpr int kSeg = 32;  // chain nodes handled per block of the forward/prox phase

inline __host__ __device__ long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

// Pack of a node: [Bbar; L] (n_k rows) then Lambda/(2 p_n) (n_v rows), both with
// the padded row stride row_stride<MT>(n_v); each matrix region is rounded to 32
// entries so every bulk copy is 16-byte aligned and a multiple of 16 bytes long.
template <typename MT>
inline __host__ __device__ long long kpad(int n_k, int n_v) { return round_up((long long)n_k * row_stride<MT>(n_v), 32); }
template <typename MT>
inline __host__ __device__ long long lpad(int n_v) { return round_up((long long)n_v * row_stride<MT>(n_v), 32); }

// Scratch for the row slices of matvec_t (same slice count as there) and for the
// per-warp block norms of the prox pass, which reuse it.
template <typename MT>
inline __host__ __device__ int part_entries(int n_v) {
  const int ld = row_stride<MT>(n_v);
  const int G = ld / (16 / (int)sizeof(MT));
  int P = kThreads / G;
  if (P > 16) P = 16;
  const int a = P * ld, b = 2 * kSeg * kWarps;
  return a > b ? a : b;
}

template <typename MT>
__host__ __device__ size_t vec_smem_bytes(int n_x, int n_u, int n_v) {
  using AT = typename Acc<MT>::T;
  const int n_k = n_x + n_u, ld = row_stride<MT>(n_v);
  size_t v = round_up((size_t)ld * sizeof(AT), 16);
  v += (size_t)(n_k + 2 * ld + part_entries<MT>(n_v) + 2 * kSeg) * sizeof(AT);
  v = round_up(v, 16);
  v += 3 * kWarps * sizeof(double) + (kSeg + 8) * sizeof(int);
  return round_up(v, 128);
}

template <typename MT>
__host__ __device__ size_t iter_smem_bytes(int S, int n_x, int n_u, int n_v, bool with_l = true) {
  size_t m = (size_t)S * (kpad<MT>(n_x + n_u, n_v) + (with_l ? lpad<MT>(n_v) : 0)) * sizeof(MT);
  m = round_up(m, 16) + 8 * sizeof(uint64_t);
  m = round_up(m, 16);
  return m + vec_smem_bytes<MT>(n_x, n_u, n_v);
}

template <typename MT>
struct Smem {
  using AT = typename Acc<MT>::T;
  unsigned char* base;  // S K-slots, then S Lambda-slots
  size_t kbytes, lbytes;
  int S;
  uint64_t* barK;  // [4]
  uint64_t* barL;  // [4]
  int ld;          // padded row stride of the matrices
  AT* dv;          // ld, 16-byte aligned, zero beyond n_v
  AT* yv;          // n_k
  AT* gv;          // ld
  AT* rv;          // ld
  AT* part;        // part_entries: mat-vec slices
  AT* red;         // aliases part: per node, per warp, the two block norms
  AT* kap;         // 2 * kSeg: per node, the prox factors kappa of the two distance blocks
  double* res3;    // 3 * kWarps
  int* seg;        // kSeg node ids
  int* flag;       // 8 ints
  __device__ MT* K(int s) const { return reinterpret_cast<MT*>(base + (size_t)s * kbytes); }
  __device__ MT* Lm(int s) const { return reinterpret_cast<MT*>(base + (size_t)S * kbytes + (size_t)s * lbytes); }
};

template <typename MT>
__device__ Smem<MT> carve(unsigned char* base, int S, int n_x, int n_u, int n_v, bool with_l = true) {
  using AT = typename Acc<MT>::T;
  Smem<MT> s;
  const int n_k = n_x + n_u;
  s.base = base;
  s.S = S;
  s.ld = row_stride<MT>(n_v);
  s.kbytes = kpad<MT>(n_k, n_v) * sizeof(MT);
  s.lbytes = with_l ? lpad<MT>(n_v) * sizeof(MT) : 0;
  size_t off = round_up((size_t)S * (s.kbytes + s.lbytes), 16);
  s.barK = reinterpret_cast<uint64_t*>(base + off);
  off += 4 * sizeof(uint64_t);
  s.barL = reinterpret_cast<uint64_t*>(base + off);
  off += 4 * sizeof(uint64_t);
  off = round_up(off, 16);
  s.dv = reinterpret_cast<AT*>(base + off);
  off += round_up((size_t)s.ld * sizeof(AT), 16);
  AT* v = reinterpret_cast<AT*>(base + off);
  s.yv = v;
  v += n_k;
  s.gv = v;
  v += s.ld;
  s.rv = v;
  v += s.ld;
  s.part = v;
  s.red = v;
  v += part_entries<MT>(n_v);
  s.kap = v;
  v += 2 * kSeg;
  off = round_up(reinterpret_cast<unsigned char*>(v) - base, 16);
  s.res3 = reinterpret_cast<double*>(base + off);
  off += 3 * kWarps * sizeof(double);
  s.seg = reinterpret_cast<int*>(base + off);
  s.flag = s.seg + kSeg;
  return s;
}

// Per-CTA cursor over the nodes of its chains, in backward (bottom-up) order.
struct Cursor {
  int chain;  // global chain index, or -1 when exhausted
  int k;      // position inside the chain (top-down index), counting down
};

// Load pipeline.  Every thread keeps an identical copy; thread 0 issues the copies.
// A load with sequence number q uses slot q % S and completes phase (q / S) of it.
struct Pipe {
  Cursor kcur, lcur;                // next chain node whose K / Lambda load is issued
  int knode, lnode;                 // thread 0: node id at kcur / lcur, loaded one issue ahead
  uint32_t kiss, kuse, liss, luse;  // issued / consumed sequence numbers
};

template <typename VT, typename MT>
struct Kern {
  using AT = typename Acc<MT>::T;
  using ST = typename St<VT>::T;  // dual state
  const IterArgs& a;
  Smem<MT>& sm;
  int S, nu, mode;
  int nd;  // dual block 2 n_x + n_u
  bool abort_ = false;
  // residual maxima in the arithmetic type (a maximum rounds nothing; float64 arithmetic
  // is slow on this GPU), power-iteration sums in float64
  AT rmax = 0, hzmax = 0, tmax = 0;
  double pnrm = 0, pdot = 0;
  unsigned long long* ttab = nullptr;  // forests with a stop per tree: the CTA's per-tree residuals

  __device__ Kern(const IterArgs& args, Smem<MT>& s, int S_, int nu_, int mode_)
      : a(args), sm(s), S(S_), nu(nu_), mode(mode_), nd(2 * args.n_x + args.n_u) {}

  __device__ ST* ys(int k) const { return reinterpret_cast<ST*>((k & 1) ? a.ybuf1 : a.ybuf0); }
  __device__ VT* wb() const { return reinterpret_cast<VT*>(a.wbuf); }
  __device__ VT* hb() const { return reinterpret_cast<VT*>(a.h); }
  __device__ const VT* cv(const void* p) const { return reinterpret_cast<const VT*>(p); }
  __device__ VT* mv(void* p) const { return reinterpret_cast<VT*>(p); }
  // Ergodic primal average (Sec. IV-A): zbar^it = (1 - theta_it) zbar^{it-1} + theta_it z^it,
  // zbar^0 = z^0 (theta_0 = 1; the previous contents are not read then).
  __device__ void ergodic_put(void* buf, long long idx, AT z, int it) const {
    VT* p = mv(buf) + idx;
    if (it == 0) {
      *p = (VT)z;
    } else {
      const AT th = (AT)a.theta[it];
      *p = (VT)(((AT)1 - th) * (AT)*p + th * z);
    }
  }
  __device__ const MT* pack(int n) const {
    return reinterpret_cast<const MT*>(a.packs) + (long long)n * a.pack_stride;
  }
  __device__ bool linear() const { return (mode & MODE_LINEAR) != 0; }
  // shared pack: the node scale 1 / (2 p_n) is applied to delta = Lambda r
  __device__ void scale_delta(int m) {
    if (!a.pscale) return;
    const AT sc = (AT)cv(a.pscale)[m];
    if (threadIdx.x < a.n_v) sm.dv[threadIdx.x] *= sc;
    __syncthreads();
  }
  // Anchored solves (bfloat16 packs): an anchor launch evaluates the solve step at
  // w_a = w^nu with the float32 packs (h_a, stored apart); the launches between run
  // the bfloat16 packs on w - w_a only, without the affine data, since the solve
  // step is affine in w: h(w) = h_a + h_lin(w - w_a).
  __device__ bool anchor() const { return (mode & MODE_ANCHOR) != 0; }
  __device__ bool delta() const { return (mode & MODE_DELTA) != 0; }
  __device__ bool no_affine() const { return (mode & (MODE_LINEAR | MODE_DELTA)) != 0; }
  __device__ bool gt() const { return (mode & MODE_GT) != 0; }
  // h of node m, entry e, as the forward sweep sees it
  __device__ AT h_at(long long m, int e) const {
    const long long q = m * a.n_k + e;
    AT v = (AT)hb()[q];
    if (a.ha) v += (AT)cv(a.ha)[q];
    return v;
  }
  // put_w with the flat index q = m n_k + e and w_a[q] loaded beforehand (delta launches)
  __device__ void put_w_at(long long q, ST w, AT wa_q) const {
    if (delta()) {
      wb()[q] = (VT)st_val(st_sub(w, st_from<ST>((double)wa_q)));
    } else {
      const VT v = (VT)st_val(w);
      wb()[q] = v;
      if (anchor()) mv(a.wa)[q] = v;
    }
  }
  // w already rounded (plain and anchor launches)
  __device__ void put_wv_at(long long q, AT w) const {
    const VT v = (VT)w;
    wb()[q] = v;
    if (anchor()) mv(a.wa)[q] = v;
  }
  // stores w^nu (entry e of node m) for the backward sweep of this launch
  __device__ void put_w(long long m, int e, ST w) const {
    const long long q = m * a.n_k + e;
    if (delta()) {
      wb()[q] = (VT)st_val(st_sub(w, st_from<ST>((double)cv(a.wa)[q])));
    } else {
      const VT v = (VT)st_val(w);
      wb()[q] = v;
      if (anchor()) mv(a.wa)[q] = v;
    }
  }

  // ---------------------------------------------------------- cursor helpers
  __device__ Cursor chain_cursor(int chain) const {
    Cursor c;
    c.chain = chain < a.n_chains ? chain : -1;
    c.k = c.chain >= 0 ? a.chain_off[c.chain + 1] - a.chain_off[c.chain] - 1 : 0;
    return c;
  }
  __device__ void advance(Cursor& c) const {
    if (c.chain < 0) return;
    if (--c.k < 0) c = chain_cursor(c.chain + gridDim.x);
  }
  __device__ int node_of(const Cursor& c) const { return a.chain_node[a.chain_off[c.chain] + c.k]; }

  // ---------------------------------------------------------- pipeline (uniform calls)
  __device__ void copy_k(uint32_t seq, int n) {
    const int slot = seq % S;
    const uint32_t bytes = (uint32_t)sm.kbytes;
    mbar_expect_tx(&sm.barK[slot], bytes);
    const unsigned char* src = reinterpret_cast<const unsigned char*>(pack(n));
    unsigned char* dst = reinterpret_cast<unsigned char*>(sm.K(slot));
    for (uint32_t o = 0; o < bytes; o += kChunk) bulk_g2s(dst + o, src + o, min((uint32_t)kChunk, bytes - o), &sm.barK[slot]);
  }
  __device__ void copy_l(uint32_t seq, int n) {
    const int slot = seq % S;
    const uint32_t bytes = (uint32_t)sm.lbytes;
    mbar_expect_tx(&sm.barL[slot], bytes);
    const unsigned char* src = reinterpret_cast<const unsigned char*>(pack(n) + kpad<MT>(a.n_k, a.n_v));
    unsigned char* dst = reinterpret_cast<unsigned char*>(sm.Lm(slot));
    for (uint32_t o = 0; o < bytes; o += kChunk) bulk_g2s(dst + o, src + o, min((uint32_t)kChunk, bytes - o), &sm.barL[slot]);
  }
  // Thread 0 reads the node id of the next copy right after issuing one, so the
  // global-memory latency of that read is spent while the node is being processed.
  __device__ void set_cursors(Pipe& p, Cursor c) {
    p.kcur = p.lcur = c;
    if (threadIdx.x == 0) p.knode = p.lnode = c.chain >= 0 ? node_of(c) : -1;
  }
  __device__ void issue_k(Pipe& p) {
    if (p.kcur.chain < 0) return;
    if (threadIdx.x == 0) {
      fence_proxy_async();
      copy_k(p.kiss, p.knode);
    }
    ++p.kiss;
    advance(p.kcur);
    if (threadIdx.x == 0 && p.kcur.chain >= 0) p.knode = node_of(p.kcur);
  }
  __device__ void issue_l(Pipe& p) {
    if (p.lcur.chain < 0) return;
    if (threadIdx.x == 0) {
      fence_proxy_async();
      copy_l(p.liss, p.lnode);
    }
    ++p.liss;
    advance(p.lcur);
    if (threadIdx.x == 0 && p.lcur.chain >= 0) p.lnode = node_of(p.lcur);
  }
  __device__ void prime(Pipe& p) {
    for (int s = 0; s < S; ++s) {
      issue_k(p);
      if (!gt()) issue_l(p);
    }
  }
  // wait for the next K (resp. Lambda) load; returns its slot; sets abort_ on timeout,
  // leaving the load counted as in flight so that drain() waits for it
  __device__ int wait_k(Pipe& p) {
    const int slot = p.kuse % S;
    const bool ok = mbar_wait(&sm.barK[slot], (p.kuse / S) & 1);
    if (__syncthreads_or(!ok)) {
      fail();
      return slot;
    }
    ++p.kuse;
    return slot;
  }
  __device__ int wait_l(Pipe& p) {
    const int slot = p.luse % S;
    const bool ok = mbar_wait(&sm.barL[slot], (p.luse / S) & 1);
    if (__syncthreads_or(!ok)) {
      fail();
      return slot;
    }
    ++p.luse;
    return slot;
  }
  // after a timeout: every copy this CTA issued lands (long bound) before it leaves
  __device__ void drain(Pipe& p) {
    for (; p.kuse < p.kiss; ++p.kuse) mbar_wait(&sm.barK[p.kuse % S], (p.kuse / S) & 1);
    for (; p.luse < p.liss; ++p.luse) mbar_wait(&sm.barL[p.luse % S], (p.luse / S) & 1);
    __syncthreads();
  }
  // let every issued copy land (bounded), forget them, and restart issuing at `next`
  __device__ void flush(Pipe& p, Cursor next) {
    bool ok = true;
    for (; p.kuse < p.kiss; ++p.kuse) ok &= mbar_wait(&sm.barK[p.kuse % S], (p.kuse / S) & 1);
    for (; p.luse < p.liss; ++p.luse) ok &= mbar_wait(&sm.barL[p.luse % S], (p.luse / S) & 1);
    set_cursors(p, next);
    if (__syncthreads_or(!ok)) fail();
  }
  __device__ void fail() {
    if (threadIdx.x == 0) a.flags[1] = SMPC_ETIMEOUT;
    abort_ = true;
  }

  // ---------------------------------------------------------- forward + prox
  // Path sums down to node `par` (inclusive) for entry e: states (V = Bbar v, X = x)
  // or inputs (U = L v).
  // Adds the nodes list[0..cnt) (top-down) to the path sums; the node ids, then their
  // vectors, are loaded 8 at a time so that the loads of a batch overlap.
  __device__ void path_add(const int* list, int cnt, int e, AT& V, AT& X, AT& U) const {
    constexpr int P = 8;
    const bool tank = e < a.n_x, lin = linear();
    for (int q0 = 0; q0 < cnt; q0 += P) {
      int id[P];
      AT hv[P], ev[P];
#pragma unroll
      for (int j = 0; j < P; ++j) id[j] = q0 + j < cnt ? list[q0 + j] : -1;
#pragma unroll
      for (int j = 0; j < P; ++j) {
        hv[j] = ev[j] = 0;
        if (id[j] >= 0) {
          hv[j] = h_at(id[j], e);
          if (tank && !lin) ev[j] = (AT)cv(a.e)[(long long)id[j] * a.n_x + e];
        }
      }
#pragma unroll
      for (int j = 0; j < P; ++j) {
        if (id[j] < 0) continue;
        if (tank) {
          V += hv[j];
          X += V + ev[j];
        } else {
          U += hv[j];
        }
      }
    }
  }
  // path sums down to top node par (inclusive) of tree `tree`, starting from its state p
  __device__ void path_init(int par, int tree, int e, AT& V, AT& X, AT& U) const {
    V = 0;
    U = 0;
    X = (e < a.n_x && !linear()) ? (AT)cv(a.p0)[(long long)tree * a.n_x + e] : (AT)0;
    if (par < 0) return;
    path_add(a.path_node + a.path_off[par], a.path_off[par + 1] - a.path_off[par], e, V, X, U);
  }

  // Forward sweep, prox, dual update and next extrapolation for the segment
  // nodes[0..len) (a chain top-down, or one top node) below node `par`.
  // Thread e owns entry e of [x (n_x); u (n_u)]: its tank's two distance-block
  // entries, or its input's box entry.  Loads are batched kB nodes at a time so
  // that their latencies overlap.
  //
  // Prox and dual update (App. C; eq. optim:dual:update1-2) without forming
  // w / lambda + x.  For a block with step lambda, set C and weight mu (mu = 0 for
  // an indicator), r = v - P_C(v) with v = w / lambda + x, and lambda r follows
  // from q = w + lambda (x - bound) (box_lr).  The distance prox moves v towards
  // P_C(v) by min(||r||, mu / lambda), so with kappa = min(1, mu / ||lambda r||)
  //   y+ = w + lambda (x - t) = kappa lambda r,   x - t = (y+ - w) / lambda.
  // Every sum that carries w runs in the state type, so y+ keeps the small move
  // lambda (x - t) however large |w| is.
  static constexpr int kB = 8;
  __device__ void phase_p(int par, const int* nodes, int len) {
    const int tree = a.tree_of[nodes[0]];
    if (!tree_active(a, tree, nu)) return;  // a forest's tree that stopped keeps its iterates
    const int e = threadIdx.x, lane = e & 31, warp = e >> 5;
    const bool tank = e < a.n_x, input = !tank && e < a.n_k;
    const int i = e - a.n_x;
    const bool lin = linear();
    const int it = nu - 1;  // iteration being finished
    const AT c = lin ? (AT)0 : (AT)a.cvec[it];
    const AT cn = lin ? (AT)0 : (AT)a.cvec[it + 1];
    ST* Y1 = ys(it);       // y^{it}
    ST* Y2 = ys(it + 1);   // y^{it-1} in, y^{it+1} out
    VT* __restrict__ Xo = mv(a.xout);
    VT* __restrict__ Uo = mv(a.uout);
    AT V = 0, X = 0, U = 0;
    if (e < a.n_k) path_init(par, a.tree_of[nodes[0]], e, V, X, U);
    const AT xs = tank ? (AT)cv(a.x_s)[e] : (AT)0;
    const AT xlo = tank ? (AT)cv(a.x_min)[e] : (AT)0;
    const AT xhi = tank ? (AT)cv(a.x_max)[e] : (AT)0;
    const AT ulo = input ? (AT)cv(a.u_min)[i] : (AT)0;
    const AT uhi = input ? (AT)cv(a.u_max)[i] : (AT)0;
    const ST zero = st_from<ST>(0.0);
    const int tank_warps = (a.n_x + 31) / 32;
    AT rm = 0, hm = 0, tm = 0;
    for (int b0 = 0; b0 < len; b0 += kSeg) {
      const int bl = min(kSeg, len - b0);
      if (e < bl) sm.seg[e] = nodes[b0 + e];
      __syncthreads();
      // pass A: forward sweep (prefix sums of h) and the two block norms ||lambda r|| per node
      for (int k0 = 0; k0 < bl; k0 += kB) {
        const int q = min(kB, bl - k0);
        AT hv[kB], ev[kB], lsv[kB], lzv[kB];
        ST s1[kB], s2[kB], z1[kB], z2[kB];
#pragma unroll
        for (int r = 0; r < kB; ++r) {
          hv[r] = ev[r] = lsv[r] = lzv[r] = 0;
          s1[r] = s2[r] = z1[r] = z2[r] = zero;
          if (r < q && e < a.n_k) {
            const int m = sm.seg[k0 + r];
            hv[r] = h_at(m, e);
            if (tank) {
              if (!lin) {
                ev[r] = (AT)cv(a.e)[(long long)m * a.n_x + e];
                const ST* y1 = Y1 + (long long)m * nd;
                const ST* y2 = Y2 + (long long)m * nd;
                s1[r] = y1[e];
                s2[r] = y2[e];
                z1[r] = y1[a.n_x + e];
                z2[r] = y2[a.n_x + e];
                lsv[r] = (AT)cv(a.step_s)[m];
                lzv[r] = (AT)cv(a.step_z)[m];
              }
            } else if (!lin) {
              ev[r] = (AT)cv(a.uhat)[(long long)m * a.n_u + i];
            }
          }
        }
#pragma unroll
        for (int r = 0; r < kB; ++r) {
          if (r < q) {
            const int m = sm.seg[k0 + r];
            AT ps = 0, pz = 0;
            if (tank) {
              V += hv[r];
              X += V + ev[r];
              Xo[(long long)m * a.n_x + e] = (VT)X;
              if (!lin) {
                const ST ws = st_extrap(s1[r], s2[r], c), wz = st_extrap(z1[r], z2[r], c);
                const ST qs = st_axpy(ws, lsv[r], X - xs);
                const AT rs = st_neg(qs) ? (AT)st_val(qs) : (AT)0;  // C = {x >= x_s}
                const AT rz = (AT)st_val(box_lr(st_axpy(wz, lzv[r], X - xhi), st_axpy(wz, lzv[r], X - xlo)));
                ps = rs * rs;
                pz = rz * rz;
              }
            } else if (input) {
              U += hv[r];
              Uo[(long long)m * a.n_u + i] = (VT)(U + ev[r]);
            }
            if (!lin && warp < tank_warps) {  // only warps holding tank entries contribute
              ps = warp_sum(ps);
              pz = warp_sum(pz);
              if (lane == 0) {
                sm.red[((k0 + r) * kWarps + warp) * 2 + 0] = ps;
                sm.red[((k0 + r) * kWarps + warp) * 2 + 1] = pz;
              }
            }
          }
        }
      }
      __syncthreads();
      if (!lin && e < bl) {  // one thread per node: kappa = min(1, mu / ||lambda r||) of both blocks
        const int m = sm.seg[e];
        AT ds2 = 0, dz2 = 0;
        for (int w = 0; w < tank_warps; ++w) {
          ds2 += sm.red[(e * kWarps + w) * 2 + 0];
          dz2 += sm.red[(e * kWarps + w) * 2 + 1];
        }
        const AT ds = sqrt(ds2), dz = sqrt(dz2);
        const AT mus = (AT)cv(a.mu_s)[m], muz = (AT)a.gamma_d;
        sm.kap[2 * e + 0] = ds > mus ? mus / ds : (AT)1;
        sm.kap[2 * e + 1] = dz > muz ? muz / dz : (AT)1;
      }
      __syncthreads();
      // pass B: prox (App. C), dual update, extrapolation w^{it+1}
      if (e < a.n_k) {
        for (int k0 = 0; k0 < bl; k0 += kB) {
          const int q = min(kB, bl - k0);
          AT zv[kB], l1[kB], l2[kB], i1[kB], i2[kB];
          ST v1[kB], v2[kB], w1[kB], w2[kB];
#pragma unroll
          for (int r = 0; r < kB; ++r) {
            zv[r] = 0;
            v1[r] = v2[r] = w1[r] = w2[r] = zero;
            l1[r] = l2[r] = i1[r] = i2[r] = 1;
            if (r < q) {
              const int m = sm.seg[k0 + r];
              const ST* y1 = Y1 + (long long)m * nd;
              const ST* y2 = Y2 + (long long)m * nd;
              if (tank) {
                zv[r] = (AT)Xo[(long long)m * a.n_x + e];
                v1[r] = y1[e];
                v2[r] = y2[e];
                w1[r] = y1[a.n_x + e];
                w2[r] = y2[a.n_x + e];
                l1[r] = (AT)cv(a.step_s)[m];
                l2[r] = (AT)cv(a.step_z)[m];
                if (!lin) {
                  i1[r] = (AT)cv(a.inv_s)[m];
                  i2[r] = (AT)cv(a.inv_z)[m];
                }
              } else {
                zv[r] = (AT)Uo[(long long)m * a.n_u + i];
                v1[r] = y1[2 * a.n_x + i];
                v2[r] = y2[2 * a.n_x + i];
                l1[r] = (AT)cv(a.step_p)[(long long)m * a.n_u + i];
                if (!lin) i1[r] = (AT)cv(a.inv_p)[(long long)m * a.n_u + i];
              }
            }
          }
#pragma unroll
          for (int r = 0; r < kB; ++r) {
            if (r >= q) continue;
            const int k = k0 + r;
            const int m = sm.seg[k];
            ST* y2 = Y2 + (long long)m * nd;
            if (lin) {
              // power iteration: y_{k+1} = -D^{1/2} H z, with D held in the step arrays
              if (tank) {
                const AT a1 = -sqrt(l1[r]) * zv[r], a2 = -sqrt(l2[r]) * zv[r];
                pdot += (double)a1 * (double)st_val(v1[r]) + (double)a2 * (double)st_val(w1[r]);
                pnrm += (double)a1 * a1 + (double)a2 * a2;
                y2[e] = st_from<ST>(a1);
                y2[a.n_x + e] = st_from<ST>(a2);
              } else {
                const AT a3 = -sqrt(l1[r]) * zv[r];
                pdot += (double)a3 * (double)st_val(v1[r]);
                pnrm += (double)a3 * a3;
                y2[2 * a.n_x + i] = st_from<ST>(a3);
              }
              continue;
            }
            const AT x = zv[r];
            if (tank) {
              const AT ks = sm.kap[2 * k + 0], kz = sm.kap[2 * k + 1];
              const ST ws = st_extrap(v1[r], v2[r], c), wz = st_extrap(w1[r], w2[r], c);
              const ST qs = st_axpy(ws, l1[r], x - xs);
              const ST ysn = st_scale(st_neg(qs) ? qs : zero, ks);
              const ST yzn = st_scale(box_lr(st_axpy(wz, l2[r], x - xhi), st_axpy(wz, l2[r], x - xlo)), kz);
              const AT es = (AT)st_val(st_sub(ysn, ws)) * i1[r];
              const AT ez = (AT)st_val(st_sub(yzn, wz)) * i2[r];
              y2[e] = ysn;
              y2[a.n_x + e] = yzn;
              put_w(m, e, st_add(st_extrap(ysn, v1[r], cn), st_extrap(yzn, w1[r], cn)));
              if (a.xbar) ergodic_put(a.xbar, (long long)m * a.n_x + e, x, it);
              rm = fmax(rm, fmax(fabs(es), fabs(ez)));
              hm = fmax(hm, fabs(x));
              tm = fmax(tm, fmax(fabs(x - es), fabs(x - ez)));
              if (!isfinite(st_val(ysn)) || !isfinite(st_val(yzn)) || !isfinite(x)) a.flags[1] = SMPC_EDIVERGED;
            } else {
              const ST wp = st_extrap(v1[r], v2[r], c);
              const ST ypn = box_lr(st_axpy(wp, l1[r], x - uhi), st_axpy(wp, l1[r], x - ulo));
              const AT ep = (AT)st_val(st_sub(ypn, wp)) * i1[r];
              y2[2 * a.n_x + i] = ypn;
              put_w(m, e, st_extrap(ypn, v1[r], cn));
              if (a.ubar) ergodic_put(a.ubar, (long long)m * a.n_u + i, x, it);
              rm = fmax(rm, fabs(ep));
              hm = fmax(hm, fabs(x));
              tm = fmax(tm, fabs(x - ep));
              if (!isfinite(st_val(ypn)) || !isfinite(x)) a.flags[1] = SMPC_EDIVERGED;
            }
          }
        }
      }
      __syncthreads();
    }
    rmax = fmax(rmax, rm);
    hzmax = fmax(hzmax, hm);
    tmax = fmax(tmax, tm);
    if (ttab && !lin) {
      const AT r_ = warp_max(rm), h_ = warp_max(hm), t_ = warp_max(tm);
      if (lane == 0) tree_res_add(a, ttab, tree, nu, (double)r_, (double)h_, (double)t_);
    }
  }

  // w^nu of the segment's nodes without a prox (first iteration, power iteration).
  __device__ void w_only(const int* nodes, int len) {
    const int e = threadIdx.x;
    if (e >= a.n_k) return;
    for (int k = 0; k < len; ++k) {
      const int m = nodes[k];
      const ST* ya = ys(nu) + (long long)m * nd;
      if (linear()) {
        const AT inv = (AT)rsqrt(a.pw[nu]);
        AT w;
        if (e < a.n_x)
          w = sqrt((AT)cv(a.step_s)[m]) * (AT)st_val(ya[e]) + sqrt((AT)cv(a.step_z)[m]) * (AT)st_val(ya[a.n_x + e]);
        else
          w = sqrt((AT)cv(a.step_p)[(long long)m * a.n_u + (e - a.n_x)]) * (AT)st_val(ya[2 * a.n_x + (e - a.n_x)]);
        wb()[(long long)m * a.n_k + e] = (VT)(w * inv);
      } else {
        const AT c = (AT)a.cvec[nu];
        const ST* yb = ys(nu + 1) + (long long)m * nd;
        if (e < a.n_x)
          put_w(m, e, st_add(st_extrap(ya[e], yb[e], c), st_extrap(ya[a.n_x + e], yb[a.n_x + e], c)));
        else
          put_w(m, e, st_extrap(ya[2 * a.n_x + (e - a.n_x)], yb[2 * a.n_x + (e - a.n_x)], c));
      }
    }
  }

  // ---------------------------------------------------------- warp-level Phase P
  // Node m alone on one warp (node-parallel schedule): lane l owns the entries
  // e = l + 32 k of [x; u].  The arithmetic of phase_p, with warp reductions only,
  // so the warps of a CTA run independent nodes without block barriers.
  static constexpr int kEPL = kThreads / 32;  // entries per lane (n_k <= kThreads)
  // x and u of node m come from the forward sweep (fwd_scan, previous launch).
  __device__ void warp_prox(int m, bool do_prox, bool do_w) {
    const int lane = threadIdx.x & 31;
    const bool lin = linear();
    AT X[kEPL], U[kEPL];  // x entries, or u (with u_hat) entries
#pragma unroll
    for (int k = 0; k < kEPL; ++k) {
      const int e = lane + 32 * k;
      X[k] = U[k] = 0;
      if (!do_prox || e >= a.n_k) continue;
      if (e < a.n_x)
        X[k] = (AT)cv(a.xout)[(long long)m * a.n_x + e];
      else
        U[k] = (AT)cv(a.uout)[(long long)m * a.n_u + (e - a.n_x)];
    }
    const ST zero = st_from<ST>(0.0);
    const long long mk = (long long)m * a.n_k;
    if (do_prox) {
      const int it = nu - 1;
      const AT c = lin ? (AT)0 : (AT)a.cvec[it];
      const AT cn = lin ? (AT)0 : (AT)a.cvec[it + 1];
      const ST* y1 = ys(it) + (long long)m * nd;
      ST* y2 = ys(it + 1) + (long long)m * nd;
      const AT ls = (AT)cv(a.step_s)[m], lz = (AT)cv(a.step_z)[m];
      if (lin) {  // power iteration: y_{k+1} = -D^{1/2} H z
#pragma unroll
        for (int k = 0; k < kEPL; ++k) {
          const int e = lane + 32 * k;
          if (e < a.n_x) {
            const AT a1 = -sqrt(ls) * X[k], a2 = -sqrt(lz) * X[k];
            pdot += (double)a1 * (double)st_val(y1[e]) + (double)a2 * (double)st_val(y1[a.n_x + e]);
            pnrm += (double)a1 * a1 + (double)a2 * a2;
            y2[e] = st_from<ST>(a1);
            y2[a.n_x + e] = st_from<ST>(a2);
          } else if (e < a.n_k) {
            const int i = e - a.n_x;
            const AT a3 = -sqrt((AT)cv(a.step_p)[(long long)m * a.n_u + i]) * U[k];
            pdot += (double)a3 * (double)st_val(y1[2 * a.n_x + i]);
            pnrm += (double)a3 * a3;
            y2[2 * a.n_x + i] = st_from<ST>(a3);
          }
        }
      } else {
        // block norms ||lambda r|| of the two distance blocks
        AT ps = 0, pz = 0;
#pragma unroll
        for (int k = 0; k < kEPL; ++k) {
          const int e = lane + 32 * k;
          if (e < a.n_x) {
            const ST ws = st_extrap(y1[e], y2[e], c), wz = st_extrap(y1[a.n_x + e], y2[a.n_x + e], c);
            const ST qs = st_axpy(ws, ls, X[k] - (AT)cv(a.x_s)[e]);
            const AT rs = st_neg(qs) ? (AT)st_val(qs) : (AT)0;
            const AT rz = (AT)st_val(box_lr(st_axpy(wz, lz, X[k] - (AT)cv(a.x_max)[e]),
                                            st_axpy(wz, lz, X[k] - (AT)cv(a.x_min)[e])));
            ps += rs * rs;
            pz += rz * rz;
          }
        }
        ps = warp_sum(ps);
        pz = warp_sum(pz);
        const AT ds = sqrt(ps), dz = sqrt(pz);
        const AT mus = (AT)cv(a.mu_s)[m], muz = (AT)a.gamma_d;
        const AT ks = ds > mus ? mus / ds : (AT)1, kz = dz > muz ? muz / dz : (AT)1;
        const AT is = (AT)cv(a.inv_s)[m], iz = (AT)cv(a.inv_z)[m];
        AT rm = 0, hm = 0, tm = 0;
#pragma unroll
        for (int k = 0; k < kEPL; ++k) {
          const int e = lane + 32 * k;
          if (e < a.n_x) {
            const AT x = X[k];
            const ST v1 = y1[e], w1 = y1[a.n_x + e];
            const ST ws = st_extrap(v1, y2[e], c), wz = st_extrap(w1, y2[a.n_x + e], c);
            const ST qs = st_axpy(ws, ls, x - (AT)cv(a.x_s)[e]);
            const ST ysn = st_scale(st_neg(qs) ? qs : zero, ks);
            const ST yzn = st_scale(box_lr(st_axpy(wz, lz, x - (AT)cv(a.x_max)[e]),
                                           st_axpy(wz, lz, x - (AT)cv(a.x_min)[e])), kz);
            const AT es = (AT)st_val(st_sub(ysn, ws)) * is;
            const AT ez = (AT)st_val(st_sub(yzn, wz)) * iz;
            y2[e] = ysn;
            y2[a.n_x + e] = yzn;
            put_w(m, e, st_add(st_extrap(ysn, v1, cn), st_extrap(yzn, w1, cn)));
            rm = fmax(rm, fmax(fabs(es), fabs(ez)));
            hm = fmax(hm, fabs(x));
            tm = fmax(tm, fmax(fabs(x - es), fabs(x - ez)));
            if (!isfinite(st_val(ysn)) || !isfinite(st_val(yzn)) || !isfinite(x)) a.flags[1] = SMPC_EDIVERGED;
          } else if (e < a.n_k) {
            const int i = e - a.n_x;
            const AT u = U[k];
            const AT lp = (AT)cv(a.step_p)[(long long)m * a.n_u + i];
            const ST p1 = y1[2 * a.n_x + i];
            const ST wp = st_extrap(p1, y2[2 * a.n_x + i], c);
            const ST ypn = box_lr(st_axpy(wp, lp, u - (AT)cv(a.u_max)[i]), st_axpy(wp, lp, u - (AT)cv(a.u_min)[i]));
            const AT ep = (AT)st_val(st_sub(ypn, wp)) * (AT)cv(a.inv_p)[(long long)m * a.n_u + i];
            y2[2 * a.n_x + i] = ypn;
            put_w(m, e, st_extrap(ypn, p1, cn));
            rm = fmax(rm, fabs(ep));
            hm = fmax(hm, fabs(u));
            tm = fmax(tm, fabs(u - ep));
            if (!isfinite(st_val(ypn)) || !isfinite(u)) a.flags[1] = SMPC_EDIVERGED;
          }
        }
        rmax = fmax(rmax, rm);
        hzmax = fmax(hzmax, hm);
        tmax = fmax(tmax, tm);
      }
    }
    if (do_w) {  // w^nu without a prox (first iteration, power iteration)
      const ST* ya = ys(nu) + (long long)m * nd;
      const ST* yb = ys(nu + 1) + (long long)m * nd;
#pragma unroll
      for (int k = 0; k < kEPL; ++k) {
        const int e = lane + 32 * k;
        if (e >= a.n_k) continue;
        if (lin) {
          const AT inv = (AT)rsqrt(a.pw[nu]);
          AT w;
          if (e < a.n_x)
            w = sqrt((AT)cv(a.step_s)[m]) * (AT)st_val(ya[e]) + sqrt((AT)cv(a.step_z)[m]) * (AT)st_val(ya[a.n_x + e]);
          else
            w = sqrt((AT)cv(a.step_p)[(long long)m * a.n_u + (e - a.n_x)]) * (AT)st_val(ya[2 * a.n_x + (e - a.n_x)]);
          wb()[mk + e] = (VT)(w * inv);
        } else {
          const AT c = (AT)a.cvec[nu];
          if (e < a.n_x)
            put_w(m, e, st_add(st_extrap(ya[e], yb[e], c), st_extrap(ya[a.n_x + e], yb[a.n_x + e], c)));
          else
            put_w(m, e, st_extrap(ya[2 * a.n_x + (e - a.n_x)], yb[2 * a.n_x + (e - a.n_x)], c));
        }
      }
    }
  }

  // The prox step of warp_prox (non-linear iterations) with the node's data staged in
  // shared memory: each lane copies its own entries by cp.async (issued back to back,
  // one wait), then the entries are processed in a rolled loop from shared memory, so
  // the launch pays one load latency per node and its code stays small.  stage: this
  // warp's region of prox_stage_bytes; bnd: x_s, x_max, x_min, u_max, u_min in shared
  // memory, kThreads apart.
  __device__ void warp_prox_staged(int m, const AT* bnd, unsigned char* stage, int tree = -1) {
    const int lane = threadIdx.x & 31;
    const int n_x = a.n_x, n_k = a.n_k, n_u = a.n_u;
    ST* Q0 = reinterpret_cast<ST*>(stage);  // y1, y2 of entry e's (first) block: n_k each
    ST* Q1 = Q0 + n_k;
    ST* Q2 = Q1 + n_k;                      // y1, y2 of a tank's second block: n_x each
    ST* Q3 = Q2 + n_x;
    VT* Z = reinterpret_cast<VT*>(Q3 + n_x);  // x or u: n_k
    VT* SP = Z + n_k;                         // step_p, 1 / step_p: n_u each
    VT* IP = SP + n_u;
    VT* WA = IP + n_u;                        // w_a (delta launches): n_k
    const int it = nu - 1;
    const ST* y1 = ys(it) + (long long)m * nd;
    ST* y2 = ys(it + 1) + (long long)m * nd;
    const long long mk = (long long)m * n_k;
    const bool dl = delta();
    for (int e = lane; e < n_k; e += 32) {
      if (e < n_x) {
        cp_async_elem(Z + e, cv(a.xout) + (long long)m * n_x + e);
        cp_async_elem(Q0 + e, y1 + e);
        cp_async_elem(Q1 + e, y2 + e);
        cp_async_elem(Q2 + e, y1 + n_x + e);
        cp_async_elem(Q3 + e, y2 + n_x + e);
      } else {
        const int i = e - n_x;
        cp_async_elem(Z + e, cv(a.uout) + (long long)m * n_u + i);
        cp_async_elem(Q0 + e, y1 + 2 * n_x + i);
        cp_async_elem(Q1 + e, y2 + 2 * n_x + i);
        cp_async_elem(SP + i, cv(a.step_p) + (long long)m * n_u + i);
        cp_async_elem(IP + i, cv(a.inv_p) + (long long)m * n_u + i);
      }
      if (dl) cp_async_elem(WA + e, cv(a.wa) + mk + e);
    }
    const AT c = (AT)a.cvec[it], cn = (AT)a.cvec[it + 1];
    const AT ls = (AT)cv(a.step_s)[m], lz = (AT)cv(a.step_z)[m];
    const AT mus = (AT)cv(a.mu_s)[m], muz = (AT)a.gamma_d;
    const AT is = (AT)cv(a.inv_s)[m], iz = (AT)cv(a.inv_z)[m];
    const ST zero = st_from<ST>(0.0);
    cp_async_wait_all();
    // block norms ||lambda r|| of the two distance blocks; the extrapolations w of a tank's
    // two blocks replace y^{it-1} in the staging (nothing else reads it) for the next pass
    AT ps = 0, pz = 0;
#pragma unroll 1
    for (int e = lane; e < n_x; e += 32) {
      const AT x = (AT)Z[e];
      const ST ws = st_extrap(Q0[e], Q1[e], c), wz = st_extrap(Q2[e], Q3[e], c);
      Q1[e] = ws;
      Q3[e] = wz;
      const ST qs = st_axpy(ws, ls, x - bnd[e]);
      const AT rs = st_neg(qs) ? (AT)st_val(qs) : (AT)0;
      const AT rz = (AT)st_val(box_lr(st_axpy(wz, lz, x - bnd[kThreads + e]), st_axpy(wz, lz, x - bnd[2 * kThreads + e])));
      ps += rs * rs;
      pz += rz * rz;
    }
    ps = warp_sum(ps);
    pz = warp_sum(pz);
    const AT ds = sqrt(ps), dz = sqrt(pz);
    const AT ks = ds > mus ? mus / ds : (AT)1, kz = dz > muz ? muz / dz : (AT)1;
    AT rm = 0, hm = 0, tm = 0;
#pragma unroll 1
    for (int e = lane; e < n_k; e += 32) {
      const AT wa_e = dl ? (AT)WA[e] : (AT)0;
      if (e < n_x) {
        const AT x = (AT)Z[e];
        const ST v1 = Q0[e], w1 = Q2[e];
        const ST ws = Q1[e], wz = Q3[e];  // written by the first pass (same lane)
        const ST qs = st_axpy(ws, ls, x - bnd[e]);
        const ST ysn = st_scale(st_neg(qs) ? qs : zero, ks);
        const ST yzn = st_scale(box_lr(st_axpy(wz, lz, x - bnd[kThreads + e]), st_axpy(wz, lz, x - bnd[2 * kThreads + e])), kz);
        const AT es = (AT)st_val(st_sub(ysn, ws)) * is;
        const AT ez = (AT)st_val(st_sub(yzn, wz)) * iz;
        y2[e] = ysn;
        y2[n_x + e] = yzn;
        if (dl)  // w - w_a must keep its own digits: the exact sum in the state type
          put_w_at(mk + e, st_add(st_extrap(ysn, v1, cn), st_extrap(yzn, w1, cn)), wa_e);
        else
          put_wv_at(mk + e, st_extrap_val(ysn, v1, cn) + st_extrap_val(yzn, w1, cn));
        if (a.xbar) ergodic_put(a.xbar, (long long)m * n_x + e, x, it);
        rm = fmax(rm, fmax(fabs(es), fabs(ez)));
        hm = fmax(hm, fabs(x));
        tm = fmax(tm, fmax(fabs(x - es), fabs(x - ez)));
        // the prox maps a non-finite v to 0, so the primal iterate is checked as well
        if (!isfinite(st_val(ysn)) || !isfinite(st_val(yzn)) || !isfinite(x)) a.flags[1] = SMPC_EDIVERGED;
      } else {
        const int i = e - n_x;
        const AT u = (AT)Z[e];
        const ST p1 = Q0[e];
        const ST wp = st_extrap(p1, Q1[e], c);
        const AT lp = (AT)SP[i];
        const ST ypn = box_lr(st_axpy(wp, lp, u - bnd[3 * kThreads + i]), st_axpy(wp, lp, u - bnd[4 * kThreads + i]));
        const AT ep = (AT)st_val(st_sub(ypn, wp)) * (AT)IP[i];
        y2[2 * n_x + i] = ypn;
        if (dl)
          put_w_at(mk + e, st_extrap(ypn, p1, cn), wa_e);
        else
          put_wv_at(mk + e, st_extrap_val(ypn, p1, cn));
        if (a.ubar) ergodic_put(a.ubar, (long long)m * n_u + i, u, it);
        rm = fmax(rm, fabs(ep));
        hm = fmax(hm, fabs(u));
        tm = fmax(tm, fabs(u - ep));
        if (!isfinite(st_val(ypn)) || !isfinite(u)) a.flags[1] = SMPC_EDIVERGED;
      }
    }
    rmax = fmax(rmax, rm);
    hzmax = fmax(hzmax, hm);
    tmax = fmax(tmax, tm);
    if (ttab && tree >= 0) {
      const AT r_ = warp_max(rm), h_ = warp_max(hm), t_ = warp_max(tm);
      if (lane == 0) tree_res_add(a, ttab, tree, nu, (double)r_, (double)h_, (double)t_);
    }
  }

  // ---------------------------------------------------------- backward sweep
  // One node's backward step with its pack in slots (K, L):
  //   r += [Bbar; L]' [s; psi];  delta = Lambda r;  h = [Bbar; L] delta.
  // On entry yv holds [s; psi] and thread j < n_v holds r_j in rreg.
  __device__ void node_backward(Pipe& p, int m, AT& rreg, bool refill) {
    const int e = threadIdx.x;
    const int ks = wait_k(p);
    if (abort_) return;
    matvec_t<MT, AT>(sm.K(ks), a.n_k, a.n_v, sm.ld, sm.yv, sm.gv, sm.part);
    if (e < a.n_v) {
      rreg += sm.gv[e];
      sm.rv[e] = rreg;
    }
    if (gt()) {  // r of every node, for the node-parallel Lambda / [Bbar; L] launch
      if (e < a.n_v) mv(a.rpub)[(long long)m * a.n_v + e] = (VT)rreg;
      if (refill) issue_k(p);
      __syncthreads();  // yv is rewritten by the next node
      return;
    }
    const int ls = wait_l(p);
    if (abort_) return;
    matvec_t<MT, AT>(sm.Lm(ls), a.n_v, a.n_v, sm.ld, sm.rv, sm.dv, sm.part);  // Lambda is symmetric
    scale_delta(m);
    if (refill) issue_l(p);
    matvec_n<MT, AT>(sm.K(ks), a.n_k, sm.ld, sm.dv, sm.yv);
    if (e < a.n_k) {
      if (anchor()) {  // h_a = h(w_a); the part on w - w_a starts at zero
        mv(a.ha)[(long long)m * a.n_k + e] = (VT)sm.yv[e];
        hb()[(long long)m * a.n_k + e] = (VT)0;
      } else {
        hb()[(long long)m * a.n_k + e] = (VT)sm.yv[e];
      }
    }
    if (refill) issue_k(p);
    __syncthreads();  // yv is rewritten by the next node
  }

  __device__ void chain_backward(Pipe& p, const int* nodes, int len) {
    const int e = threadIdx.x;
    AT sreg = 0, rreg = 0;
    const bool lin = no_affine();
    int m = nodes[len - 1];
    AT wcur = e < a.n_k ? (AT)wb()[(long long)m * a.n_k + e] : (AT)0;
    AT bcur = (e < a.n_v && !lin) ? (AT)cv(a.beta)[(long long)m * a.n_v + e] : (AT)0;
    for (int k = len - 1; k >= 0; --k) {
      m = nodes[k];
      AT wnext = 0, bnext = 0;
      if (k > 0) {  // prefetch the next node's vectors into registers
        const int mn = nodes[k - 1];
        if (e < a.n_k) wnext = (AT)wb()[(long long)mn * a.n_k + e];
        if (e < a.n_v && !lin) bnext = (AT)cv(a.beta)[(long long)mn * a.n_v + e];
      }
      if (e < a.n_x) {
        sreg += wcur;
        sm.yv[e] = sreg;
      } else if (e < a.n_k) {
        sm.yv[e] = wcur;
      }
      rreg += bcur;
      node_backward(p, m, rreg, true);
      if (abort_) return;
      wcur = wnext;
      bcur = bnext;
    }
    const int head = nodes[0];
    if (e < a.n_x) mv(a.spub)[(long long)head * a.n_x + e] = (VT)sreg;
    if (e < a.n_v) mv(a.rpub)[(long long)head * a.n_v + e] = (VT)rreg;
  }

  // Arrival at top node t (children and its own Phase P count); true for the last one.
  // The block barrier then one fence by thread 0 publish the whole CTA's writes (spub,
  // rpub, h, wbuf) before the arrival; the fence after the last arrival orders the reads
  // of the children's results (ld.cg) after it.
  __device__ bool arrive(int t) {
    __syncthreads();
    if (threadIdx.x == 0) {
      fence_acq_rel_gpu();
      const int old = atomicAdd(&a.counters[t], 1);
      const int last = (old == a.top_expect[t] - 1);
      if (last) {
        a.counters[t] = 0;  // nobody else touches it again in this launch
        fence_acq_rel_gpu();
      }
      sm.flag[0] = last;
    }
    __syncthreads();
    return sm.flag[0] != 0;
  }

  // Process top node t (this CTA arrived last) and climb while it stays last.
  // The chain prefetch in flight is flushed and re-issued from `next` afterwards.
  __device__ void process_top(Pipe& p, int t, Cursor next) {
    flush(p, next);
    if (abort_) return;
    const int e = threadIdx.x;
    const bool lin = no_affine();
    while (t >= 0) {
      if (threadIdx.x == 0) {
        fence_proxy_async();
        copy_k(p.kiss, t);
        if (!gt()) copy_l(p.liss, t);
      }
      ++p.kiss;
      if (!gt()) ++p.liss;
      const int cb = a.child_begin[t], cc = a.child_count[t];
      AT sreg = 0, rreg = 0;
      if (e < a.n_k) {
        AT v = (AT)ldcg(wb() + (long long)t * a.n_k + e);
        if (e < a.n_x) {
          for (int c = cb; c < cb + cc; ++c) v += (AT)ldcg(mv(a.spub) + (long long)c * a.n_x + e);
          sreg = v;
        }
        sm.yv[e] = v;
      }
      if (e < a.n_v) {
        rreg = lin ? (AT)0 : (AT)cv(a.beta)[(long long)t * a.n_v + e];
        for (int c = cb; c < cb + cc; ++c) rreg += (AT)ldcg(mv(a.rpub) + (long long)c * a.n_v + e);
      }
      node_backward(p, t, rreg, false);
      if (abort_) return;
      if (e < a.n_x) mv(a.spub)[(long long)t * a.n_x + e] = (VT)sreg;
      if (e < a.n_v) mv(a.rpub)[(long long)t * a.n_v + e] = (VT)rreg;
      t = a.parent[t];
      if (t < 0 || !arrive(t)) break;
    }
    prime(p);
  }

  // ---------------------------------------------------------- the launch
  __device__ void run() {
    const int tid = threadIdx.x;
    const bool do_prox = (mode & MODE_PROX) != 0 && nu >= 1;
    const bool do_bwd = (mode & MODE_BWD) != 0;

    Pipe p;
    set_cursors(p, chain_cursor(blockIdx.x));
    p.kiss = p.kuse = p.liss = p.luse = 0;
    for (int j = a.n_v + tid; j < sm.ld; j += kThreads) sm.dv[j] = 0;
    if (tid == 0) {
      for (int s = 0; s < S; ++s) {
        mbar_init(&sm.barK[s], 1);
        mbar_init(&sm.barL[s], 1);
      }
      fence_barrier_init();
      fence_proxy_async();
    }
    __syncthreads();
    if (do_bwd) prime(p);

    // top-node tasks: forward + prox (Phase P) or w only, then the arrival
    for (int ti = blockIdx.x; ti < a.n_top && !abort_; ti += gridDim.x) {
      const int t = a.top_nodes[ti];
      if (do_prox) phase_p(a.parent[t], a.top_nodes + ti, 1);
      if (do_bwd) {
        if ((!do_prox || linear()) && !(mode & MODE_WREADY)) {
          w_only(a.top_nodes + ti, 1);
          __syncthreads();
        }
        if (arrive(t)) process_top(p, t, chain_cursor(blockIdx.x));
      }
    }

    // chains
    for (int ch = blockIdx.x; ch < a.n_chains && !abort_; ch += gridDim.x) {
      const int cb = a.chain_off[ch], len = a.chain_off[ch + 1] - cb;
      const int* nodes = a.chain_node + cb;
      if (do_prox) phase_p(a.chain_parent[ch], nodes, len);
      if (!do_bwd) continue;
      if ((!do_prox || linear()) && !(mode & MODE_WREADY)) {
        w_only(nodes, len);
        __syncthreads();
      }
      chain_backward(p, nodes, len);
      if (abort_) break;
      const int par = a.chain_parent[ch];
      if (mode & MODE_NOCLIMB) continue;  // a shard: the heads' s and r go to the exchange
      if (par >= 0 && arrive(par)) process_top(p, par, chain_cursor(ch + gridDim.x));
    }

    if (abort_) drain(p);
    reduce_out(do_prox);
  }

  // per-CTA reductions: residual maxima (Sec. IV-E) or power-iteration sums
  __device__ void reduce_out(bool do_prox) {
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    if (do_prox && !linear()) {
      const AT r = warp_max(rmax), hz = warp_max(hzmax), tt = warp_max(tmax);
      AT* r3 = reinterpret_cast<AT*>(sm.res3);  // 3 kWarps entries fit in its 3 kWarps doubles
      if (lane == 0) {
        r3[warp] = r;
        r3[kWarps + warp] = hz;
        r3[2 * kWarps + warp] = tt;
      }
      __syncthreads();
      if (tid == 0) {
        AT R = 0, HZ = 0, TT = 0;
        for (int w = 0; w < kWarps; ++w) {
          R = fmax(R, r3[w]);
          HZ = fmax(HZ, r3[kWarps + w]);
          TT = fmax(TT, r3[2 * kWarps + w]);
        }
        unsigned long long* slot = a.res + 3ll * (nu - 1);
        atomic_max_nonneg(slot + 0, (double)R);
        atomic_max_nonneg(slot + 1, (double)HZ);
        atomic_max_nonneg(slot + 2, (double)TT);
      }
    } else if (do_prox && linear()) {
      const double nr = warp_sum(pnrm), dt = warp_sum(pdot);
      if (lane == 0) {
        sm.res3[warp] = nr;
        sm.res3[kWarps + warp] = dt;
      }
      __syncthreads();
      if (tid == 0) {
        double NR = 0, DT = 0;
        for (int w = 0; w < kWarps; ++w) {
          NR += sm.res3[w];
          DT += sm.res3[kWarps + w];
        }
        atomicAdd(&a.pw[nu], NR);
        atomicAdd(&a.pw[a.pw_len + nu - 1], DT);
      }
    }
  }
};

// Uniform early exit of a launch of iteration nu: the solve stopped or failed, or (with
// `decide`) the residual of iteration nu - 2 met the tolerance, which ends the solve
// after nu - 1 iterations.
__device__ bool early_exit(const IterArgs& a, int nu, int mode, int* flag, bool decide) {
  if (threadIdx.x == 0) {
    int stop = 0;
    if (mode & MODE_CHECK) {
      // the flags and the residuals are loaded together (one round trip)
      const bool test = decide && a.tol > 0 && nu >= 2;
      const unsigned long long* r = a.res + 3ll * (test ? nu - 2 : 0);
      const int done = ldcg(a.flags + 0), err = ldcg(a.flags + 1);
      unsigned long long r0 = 0, r1 = 0, r2 = 0;
      if (test) {
        r0 = ldcg(r + 0);
        r1 = ldcg(r + 1);
        r2 = ldcg(r + 2);
      }
      if (done >= 0 || err != 0) stop = 1;
      if (test && !stop && !a.res_tree) {
        const double rho = __longlong_as_double((long long)r0);
        const double hz = __longlong_as_double((long long)r1);
        const double tt = __longlong_as_double((long long)r2);
        if (rho / (1.0 + fmax(hz, tt)) <= a.tol) {
          stop = 1;
          if (blockIdx.x == 0) a.flags[0] = nu - 1;
        }
      }
    }
    *flag = stop;
  }
  __syncthreads();
  if (*flag == 0 && (mode & MODE_CHECK) && decide && a.res_tree && a.tol > 0 && nu >= 2) {
    // a stop per tree: block 0 records the trees that stop at this launch; the solve ends
    // when every tree has stopped (each CTA reaches the same answer)
    bool all = true;
    for (int r = threadIdx.x; r < a.R; r += blockDim.x) {
      const bool was = ldcg(a.tree_done + r) >= 0;
      const bool now = !was && tree_stops(a.res_tree + 3ll * ((long long)(nu - 2) * a.R + r), a.tol);
      if (now && blockIdx.x == 0) a.tree_done[r] = nu - 1;
      all = all && (was || now);
    }
    all = __syncthreads_and(all);
    if (all) {
      if (blockIdx.x == 0 && threadIdx.x == 0) a.flags[0] = nu - 1;
      return true;
    }
  }
  return *flag != 0;
}

template <typename VT, typename MT>
__global__ void __launch_bounds__(kThreads, 1)
    apg_iter(const __grid_constant__ IterArgs a, int S, int nu, int mode) {
  grid_dep_sync();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ unsigned long long ttab[3 * kTreeTable];
  Smem<MT> sm = carve<MT>(smem_raw, S, a.n_x, a.n_u, a.n_v);
  if (early_exit(a, nu, mode, sm.flag + 1, true)) return;
  Kern<VT, MT> k(a, sm, S, nu, mode);
  const bool tabled = a.res_tree && (mode & MODE_PROX) && nu >= 1 && !(mode & MODE_LINEAR);
  if (tabled) {
    tree_table_clear(a, ttab);
    __syncthreads();
    k.ttab = ttab;
  }
  k.run();
  if (tabled) {
    __syncthreads();
    tree_table_flush(a, ttab, nu);
  }
}

// ------------------------------------------------------------------ fused backward pass (schedule 4)
// The whole backward sweep of Algorithm 1 in one launch with every pack read once: one CTA
// of kBT threads per chain (and the top nodes by last arrival, as in apg_iter), each chain
// node's pack [Bbar; L | Lambda / (2 p_n)] streamed through S shared-memory slots with
// cp.async.bulk while the previous nodes are processed.  Per node, three mat-vecs from
// shared memory: g = [Bbar; L]' [s; psi], r = r_below + beta + g, delta = Lambda r, and
// h = [Bbar; L] delta.  512 threads per CTA (one CTA per SM) halve each mat-vec's serial
// work against apg_iter's 256, which keeps the node time below the pack's HBM time.
constexpr int kBT = 512;

template <typename MT>
__host__ __device__ inline int bwd_slices(int n_v) {
  const int G = row_stride<MT>(n_v) / (16 / (int)sizeof(MT));
  const int P = kBT / G;
  return P > 20 ? 20 : P;
}


template <typename MT>
__host__ __device__ inline size_t bwd_smem_bytes(int S, int n_x, int n_u, int n_v) {
  using AT = typename Acc<MT>::T;
  const int n_k = n_x + n_u, ld = row_stride<MT>(n_v);
  size_t m = (size_t)S * (kpad<MT>(n_k, n_v) + lpad<MT>(n_v)) * sizeof(MT);
  m = round_up(m, 16) + 4 * sizeof(uint64_t);
  m = round_up(m, 16);
  m += ((size_t)3 * ld + round_up(n_k, 4) + (size_t)bwd_slices<MT>(n_v) * ld) * sizeof(AT);
  m = round_up(m, 16) + 16 * sizeof(int);
  return round_up(m, 128);
}

template <typename VT, typename MT>
struct Bwd {
  using AT = typename Acc<MT>::T;
  const IterArgs& a;
  int S, nu, mode, ld;
  unsigned char* base;
  size_t kbytes, lbytes;
  uint64_t* bar;  // one per slot: the node's [Bbar; L] and Lambda copies
  AT *dv, *rv, *gv, *yv, *part;
  int* flag;
  uint32_t iss = 0, use = 0;  // loads issued / consumed (the same in every thread)
  // next chain node to load: chain, position k (counting down) and the chain's first entry
  // in chain_node, so that a node id is one load whose latency is spent while a node runs
  struct Cur {
    int chain, k, off;
  } cur;
  int cnode = -1;             // thread 0: the node id at cur
  bool abort_ = false;
  bool pending_ = false;  // the previous node's slot is to be refilled at the next B1

  __device__ Bwd(const IterArgs& args, unsigned char* smem, int S_, int nu_, int mode_)
      : a(args), S(S_), nu(nu_), mode(mode_), base(smem) {
    ld = row_stride<MT>(a.n_v);
    kbytes = kpad<MT>(a.n_k, a.n_v) * sizeof(MT);
    lbytes = lpad<MT>(a.n_v) * sizeof(MT);
    size_t off = round_up((size_t)S * (kbytes + lbytes), 16);
    bar = reinterpret_cast<uint64_t*>(base + off);
    off = round_up(off + 4 * sizeof(uint64_t), 16);
    AT* v = reinterpret_cast<AT*>(base + off);
    dv = v;
    v += ld;
    rv = v;
    v += ld;
    gv = v;
    v += ld;
    yv = v;
    v += round_up(a.n_k, 4);
    part = v;
    v += bwd_slices<MT>(a.n_v) * ld;
    off = round_up(reinterpret_cast<unsigned char*>(v) - base, 16);
    flag = reinterpret_cast<int*>(base + off);
  }
  __device__ MT* K(int s) const { return reinterpret_cast<MT*>(base + (size_t)s * (kbytes + lbytes)); }
  __device__ MT* Lm(int s) const { return reinterpret_cast<MT*>(base + (size_t)s * (kbytes + lbytes) + kbytes); }
  __device__ const MT* pack(int n) const {
    return reinterpret_cast<const MT*>(a.packs) + (long long)n * a.pack_stride;
  }
  __device__ const VT* cv(const void* p) const { return reinterpret_cast<const VT*>(p); }
  __device__ VT* mv(void* p) const { return reinterpret_cast<VT*>(p); }
  __device__ bool no_affine() const { return (mode & (MODE_LINEAR | MODE_DELTA)) != 0; }

  // ---------------------------------------------------------- pipeline
  __device__ Cur chain_cursor(int chain) const {
    Cur c;
    c.chain = chain < a.n_chains ? chain : -1;
    c.off = c.chain >= 0 ? a.chain_off[c.chain] : 0;
    c.k = c.chain >= 0 ? a.chain_off[c.chain + 1] - c.off - 1 : 0;
    return c;
  }
  __device__ void advance(Cur& c) const {
    if (c.chain < 0) return;
    if (--c.k < 0) c = chain_cursor(c.chain + gridDim.x);
  }
  __device__ int node_of(const Cur& c) const { return a.chain_node[c.off + c.k]; }
  __device__ void copy_node(uint32_t seq, int n) {  // thread 0
    const int slot = seq % S;
    fence_proxy_async();
    mbar_expect_tx(&bar[slot], (uint32_t)(kbytes + lbytes));
    const unsigned char* src = reinterpret_cast<const unsigned char*>(pack(n));
    bulk_g2s(K(slot), src, (uint32_t)kbytes, &bar[slot]);
    bulk_g2s(Lm(slot), src + kpad<MT>(a.n_k, a.n_v) * sizeof(MT), (uint32_t)lbytes, &bar[slot]);
  }
  __device__ void set_cursor(Cur c) {
    cur = c;
    if (threadIdx.x == 0) cnode = c.chain >= 0 ? node_of(c) : -1;
  }
  __device__ void issue() {
    if (cur.chain < 0) return;
    if (threadIdx.x == 0) copy_node(iss, cnode);
    ++iss;
    advance(cur);
    if (threadIdx.x == 0 && cur.chain >= 0) cnode = node_of(cur);  // used at the next issue
  }
  __device__ void prime() {
    for (int q = 0; q < S; ++q) issue();
  }
  __device__ void fail() {
    if (threadIdx.x == 0) a.flags[1] = SMPC_ETIMEOUT;
    abort_ = true;
  }
  __device__ void drain() {
    for (; use < iss; ++use) mbar_wait(&bar[use % S], (use / S) & 1);
    __syncthreads();
  }
  // let every issued load land (bounded) and restart issuing at `next`
  __device__ void flush(Cur next) {
    bool ok = true;
    for (; use < iss; ++use) ok &= mbar_wait(&bar[use % S], (use / S) & 1);
    set_cursor(next);
    if (__syncthreads_or(!ok)) fail();
  }

  // ---------------------------------------------------------- mat-vecs from shared memory
  // Partial column sums of A' x (A with R rows): thread (g, p) accumulates columns
  // g V .. g V + V - 1 over the p-th row slice and stores them with one vector store into
  // part (slice p, row stride ld); node_step adds the slices in a fixed order.
  __device__ void mtv_t_part(const MT* A, int R, const AT* x) {
    constexpr int V = Vec<MT>::V;
    const int t = threadIdx.x;
    const int G = ld / V;
    const int P = bwd_slices<MT>(a.n_v);
    const int rc = (R + P - 1) / P;
    if (t >= P * G) return;
    const int g = t % G, p = t / G;
    const int i0 = p * rc, i1 = min(R, i0 + rc);
    AT acc[V];
#pragma unroll
    for (int k = 0; k < V; ++k) acc[k] = 0;
    const MT* col = A + g * V;
#pragma unroll 4
    for (int i = i0; i < i1; ++i) {
      AT av[V];
      ld16(col + (long long)i * ld, av);
      const AT xi = x[i];
#pragma unroll
      for (int k = 0; k < V; ++k) acc[k] += av[k] * xi;
    }
    st16(part + p * ld + g * V, acc);
  }
  // put(i, A_i . x) for the rows i < R of A (row stride ld; x zero beyond its entries up
  // to ld), Q lanes per row (Q = 2 or 4) and NR rows per lane (1 or 2).  A warp takes
  // NR * 32 / Q consecutive rows per pass: lane l has rows r, r + 32 / Q, ... of them,
  // r = l mod 32/Q, and the part q = l div (32/Q) of their 16-byte groups (q, q + Q, ...).
  // The eight lanes of a load phase read eight different rows (no bank conflicts) and the
  // same piece of x (a broadcast), which serves all NR rows of the lane; the Q parts are
  // added by shuffles in a fixed order.
  template <int Q, int NR, typename F>
  __device__ void mv_rows(const MT* A, int R, const AT* x, F&& put) {
    constexpr int V = Vec<MT>::V, RW = 32 / Q;
    const int G = ld / V;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = lane / RW;
    for (int i0 = NR * RW * warp; i0 < R; i0 += NR * RW * (kBT / 32)) {  // warp-uniform
      const int i = i0 + lane % RW;
      AT acc[NR][2];
      const MT* row[NR];
#pragma unroll
      for (int n = 0; n < NR; ++n) {
        acc[n][0] = acc[n][1] = 0;
        const int in = i + n * RW;
        row[n] = A + (long long)(in < R ? in : i) * ld;
      }
      if (i < R) {
#pragma unroll 2
        for (int g = q; g < G; g += Q) {
          AT xv[V];
          ldx(x + g * V, xv);
#pragma unroll
          for (int n = 0; n < NR; ++n) {
            AT av[V];
            ld16(row[n] + g * V, av);
#pragma unroll
            for (int k = 0; k < V; k += 2) {
              acc[n][0] += av[k] * xv[k];
              acc[n][1] += av[k + 1] * xv[k + 1];
            }
          }
        }
      }
#pragma unroll
      for (int n = 0; n < NR; ++n) {
        AT v = acc[n][0] + acc[n][1];
#pragma unroll
        for (int d = RW; d < 32; d *= 2) v += __shfl_xor_sync(0xffffffffu, v, d);
        const int in = i + n * RW;
        if (q == 0 && in < R) put(in, v);
      }
    }
  }
  // rows per lane of the row dots: two where a matrix entry is four or eight bytes (the
  // vector loads are then shared), one for bfloat16 (whose row dots are shorter)
  static constexpr int kNR = sizeof(MT) >= 4 ? 2 : 1;

  // ---------------------------------------------------------- one node's backward step
  // On entry yv holds [s; psi] of node m (visible to every thread) and thread j < n_v holds
  // r_j (the children's r and beta) in rreg.  Three block barriers:
  //   P1 partial column sums of g = [Bbar; L]' [s; psi]     | B1 (then the previous node's
  //                                                          |    slot is refilled)
  //   P2 r = rreg + g (thread j); yv <- the next chain node's [s; psi] (when has_next), and
  //      rreg += its beta after r is published              | B2
  //   P3 delta = Lambda r (row dots; Lambda is symmetric)    | B3
  //   P4 h = [Bbar; L] delta to global memory.
  // The slot's arrival is awaited by each thread before P1; a timeout is agreed on at B1.
  // With refill, this node's slot is refilled at the next node's B1, or by the caller
  // (at once behind a fourth barrier when there is one slot).
  __device__ void node_step(int m, AT& rreg, AT& sreg, bool has_next, AT wnext, AT bnext, bool refill) {
    const int t = threadIdx.x;
    const int slot = use % S;
    const bool ok = mbar_wait(&bar[slot], (use / S) & 1);
    mtv_t_part(K(slot), a.n_k, yv);
    if (__syncthreads_or(!ok)) {  // B1
      fail();
      return;
    }
    ++use;
    if (pending_) {  // the previous node's slot: its last reads (P4) ended before B1
      issue();
      pending_ = false;
    }
    if (t < a.n_v) {
      const int P = bwd_slices<MT>(a.n_v);
      AT v[20];
#pragma unroll
      for (int p = 0; p < 20; ++p) v[p] = p < P ? part[p * ld + t] : (AT)0;
      AT s0 = 0, s1 = 0;
#pragma unroll
      for (int p = 0; p < 20; p += 2) {  // fixed order: deterministic
        s0 += v[p];
        s1 += v[p + 1];
      }
      rreg += s0 + s1;
      rv[t] = rreg;
      if (has_next) rreg += bnext;
    }
    if (has_next) {
      if (t < a.n_x) {
        sreg += wnext;
        yv[t] = sreg;
      } else if (t < a.n_k) {
        yv[t] = wnext;
      }
    }
    __syncthreads();  // B2
    const AT sc = a.pscale ? (AT)cv(a.pscale)[m] : (AT)1;  // shared pack: delta = (Lambda r) / (2 p_n)
    mv_rows<4, kNR>(Lm(slot), a.n_v, rv, [&](int i, AT v) { dv[i] = v * sc; });
    __syncthreads();  // B3
    const long long q0 = (long long)m * a.n_k;
    const bool anchor = (mode & MODE_ANCHOR) != 0;
    mv_rows<kNR == 2 ? 4 : 2, kNR>(K(slot), a.n_k, dv, [&](int i, AT v) {
      if (anchor) {  // h_a = h(w_a); the part on w - w_a starts at zero
        mv(a.ha)[q0 + i] = (VT)v;
        mv(a.h)[q0 + i] = (VT)0;
      } else {
        mv(a.h)[q0 + i] = (VT)v;
      }
    });
    if (refill && S == 1) {  // one slot: the next node needs it, refill now
      __syncthreads();
      issue();
    } else {
      pending_ = refill;  // the slot is refilled at the next node's B1 (or at the chain's end)
    }
  }

  // The ids a chain starts with (offset, length, bottom node, the node above it),
  // loaded one chain ahead so that no chain start waits for dependent global loads.
  struct ChainIds {
    int cb, len, m0, m1;
  };
  __device__ ChainIds chain_ids(int ch) const {
    ChainIds c{0, 0, -1, -1};
    if (ch < a.n_chains) {
      c.cb = a.chain_off[ch];
      c.len = a.chain_off[ch + 1] - c.cb;
      c.m0 = a.chain_node[c.cb + c.len - 1];
      c.m1 = c.len > 1 ? a.chain_node[c.cb + c.len - 2] : -1;
    }
    return c;
  }
  // w and beta entries of thread e for node m (beta zero for the linear modes)
  __device__ void node_vectors(int m, AT& w, AT& b) const {
    const int e = threadIdx.x;
    w = e < a.n_k ? (AT)cv(a.wbuf)[(long long)m * a.n_k + e] : (AT)0;
    b = (e < a.n_v && !no_affine()) ? (AT)cv(a.beta)[(long long)m * a.n_v + e] : (AT)0;
  }

  // Chain c bottom-up.  wpre, bpre: on entry the bottom node's w and beta entries; on
  // return those of the next chain's bottom node nx.m0 (loaded during the last node).
  // Node ids are loaded two nodes ahead and each node's vectors one node ahead.
  __device__ void chain(const ChainIds& c, const ChainIds& nx, AT& wpre, AT& bpre) {
    const int e = threadIdx.x;
    const int* gn = a.chain_node + c.cb;
    AT sreg = 0, rreg = bpre;
    __syncthreads();  // the previous node step's reads of yv are done
    if (e < a.n_x) {
      sreg = wpre;
      yv[e] = wpre;
    } else if (e < a.n_k) {
      yv[e] = wpre;
    }
    __syncthreads();
    int m = c.m0, m1 = c.m1, head = c.m0;
    for (int k = c.len - 1; k >= 0; --k) {
      const int m2 = k >= 2 ? gn[k - 2] : -1;
      AT wnext = 0, bnext = 0;
      if (k > 0)
        node_vectors(m1, wnext, bnext);  // the next node's, while this node runs
      else if (nx.m0 >= 0)
        node_vectors(nx.m0, wpre, bpre);  // the next chain's bottom node
      head = m;
      node_step(m, rreg, sreg, k > 0, wnext, bnext, true);
      if (abort_) return;
      m = m1;
      m1 = m2;
    }
    if (pending_) {  // the last node's slot
      __syncthreads();
      issue();
      pending_ = false;
    }
    if (e < a.n_x) mv(a.spub)[(long long)head * a.n_x + e] = (VT)sreg;
    if (e < a.n_v) mv(a.rpub)[(long long)head * a.n_v + e] = (VT)rreg;
  }

  // arrival at top node t (its children and its own ready w count); true for the last one
  __device__ bool arrive(int t) {
    __syncthreads();
    if (threadIdx.x == 0) {
      fence_acq_rel_gpu();
      const int old = atomicAdd(&a.counters[t], 1);
      const int last = (old == a.top_expect[t] - 1);
      if (last) {
        a.counters[t] = 0;
        fence_acq_rel_gpu();
      }
      flag[0] = last;
    }
    __syncthreads();
    return flag[0] != 0;
  }

  // top node t (this CTA arrived last), then up while it stays last
  __device__ void process_top(int t, Cur next) {
    flush(next);
    if (abort_) return;
    const int e = threadIdx.x;
    const bool lin = no_affine();
    while (t >= 0) {
      if (threadIdx.x == 0) copy_node(iss, t);
      ++iss;
      const int cb = a.child_begin[t], cc = a.child_count[t];
      AT sreg = 0, rreg = 0;
      if (e < a.n_k) {
        AT v = (AT)ldcg(cv(a.wbuf) + (long long)t * a.n_k + e);
        if (e < a.n_x) {
          for (int c = cb; c < cb + cc; ++c) v += (AT)ldcg(cv(a.spub) + (long long)c * a.n_x + e);
          sreg = v;
        }
        yv[e] = v;
      }
      if (e < a.n_v) {
        rreg = lin ? (AT)0 : (AT)cv(a.beta)[(long long)t * a.n_v + e];
        for (int c = cb; c < cb + cc; ++c) rreg += (AT)ldcg(cv(a.rpub) + (long long)c * a.n_v + e);
      }
      __syncthreads();  // yv is complete
      node_step(t, rreg, sreg, false, (AT)0, (AT)0, false);
      if (abort_) return;
      if (e < a.n_x) mv(a.spub)[(long long)t * a.n_x + e] = (VT)sreg;
      if (e < a.n_v) mv(a.rpub)[(long long)t * a.n_v + e] = (VT)rreg;
      t = a.parent[t];
      if (t < 0 || !arrive(t)) break;
    }
    prime();
  }

  __device__ void run() {
    const int tid = threadIdx.x;
    for (int j = a.n_v + tid; j < ld; j += kBT) dv[j] = rv[j] = 0;  // the row dots read x up to ld
    if (tid == 0) {
      for (int q = 0; q < S; ++q) mbar_init(&bar[q], 1);
      fence_barrier_init();
      fence_proxy_async();
    }
    __syncthreads();
    set_cursor(chain_cursor(blockIdx.x));
    prime();
    for (int ti = blockIdx.x; ti < a.n_top && !abort_; ti += gridDim.x) {
      const int t = a.top_nodes[ti];
      if (arrive(t)) process_top(t, chain_cursor(blockIdx.x));
    }
    ChainIds c = chain_ids(blockIdx.x);
    AT wpre = 0, bpre = 0;
    if (c.m0 >= 0) node_vectors(c.m0, wpre, bpre);
    for (int ch = blockIdx.x; ch < a.n_chains && !abort_; ch += gridDim.x) {
      const int par = a.chain_parent[ch];  // read now, used after the chain
      const ChainIds nx = chain_ids(ch + gridDim.x);
      chain(c, nx, wpre, bpre);
      if (abort_) break;
      c = nx;
      if (mode & MODE_NOCLIMB) continue;
      if (par >= 0 && arrive(par)) process_top(par, chain_cursor(ch + gridDim.x));
    }
    if (abort_) drain();
  }
};

template <typename VT, typename MT>
__global__ void __launch_bounds__(kBT, 1)
    chain_bwd(const __grid_constant__ IterArgs a, int S, int nu, int mode) {
  grid_dep_sync();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int flag[2];
  if (early_exit(a, nu, mode, flag, false)) return;
  Bwd<VT, MT> k(a, smem_raw, S, nu, mode);
  k.run();
}

// ------------------------------------------------------------------ node-parallel schedule
// The backward sweep is linear in (w, beta).  With s = subtree sums of xi,
// g_n = [Bbar; L]_n' [s_n; psi_n] and r = subtree sums of beta + g, the mat-vecs of
// different nodes are independent, so one iteration becomes five launches:
//   prox_node  forward sweep (each node sums its own path), prox, dual update, w^nu
//   scan (s)   s_n = xi_n + sum_c s_c             (chains bottom-up, top nodes on arrival)
//   node_gt    g_n = [Bbar; L]_n' [s_n; psi_n]
//   scan (r)   r_n = beta_n + g_n + sum_c r_c      (in place over g)
//   node_dh    h_n = [Bbar; L]_n (Lambda_n / (2 p_n)) r_n
// [Bbar; L] is read twice per iteration instead of once, but each launch has one
// independent task per node instead of one sequential task per chain.

// Forward sweep of iteration nu - 1: one CTA per segment (a top node with its path
// from the root, or a chain with the path above it).  The vectors (h, h_a, e or u_hat)
// of up to fwd_chunk nodes are staged in shared memory by cp.async, issued back to
// back with one wait, so a chunk costs about one load latency; thread e then sums
// entry e down the chunk from shared memory (it reads only what it copied itself)
// and stores x (tank entries) or u (inputs) of the segment's own nodes.
template <typename VT>
__host__ __device__ constexpr int fwd_chunk() { return sizeof(VT) == 4 ? 32 : 16; }
// h and e (or u_hat) of a chunk, and h_a behind them for anchored solves only, so that
// plain solves fit one more CTA per SM
template <typename VT>
size_t fwd_smem_bytes(int n_k, bool anchored) { return (size_t)(anchored ? 3 : 2) * fwd_chunk<VT>() * n_k * sizeof(VT); }

template <typename VT, typename MT>
__global__ void __launch_bounds__(kThreads) fwd_scan(const __grid_constant__ IterArgs a, int nu, int mode) {
  grid_dep_sync();
  using AT = typename Acc<MT>::T;
  constexpr int KC = fwd_chunk<VT>();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int flag[2];
  __shared__ int sid[KC];
  __shared__ AT sX[kThreads];  // general A: the parent's state
  if (early_exit(a, nu, mode, flag, true)) return;
  const int n_k = a.n_k, e = threadIdx.x, i = e - a.n_x;
  const bool act = e < n_k, tank = e < a.n_x, lin = (mode & MODE_LINEAR) != 0;
  VT* sh = reinterpret_cast<VT*>(smem_raw);  // KC x n_k each: h, e or u_hat, h_a (anchored solves)
  VT* se = sh + KC * n_k;
  VT* sa = se + KC * n_k;
  const VT* H = reinterpret_cast<const VT*>(a.h);
  const VT* HA = reinterpret_cast<const VT*>(a.ha);
  const VT* E = reinterpret_cast<const VT*>(a.e);
  const VT* UH = reinterpret_cast<const VT*>(a.uhat);
  VT* XO = reinterpret_cast<VT*>(a.xout);
  VT* UO = reinterpret_cast<VT*>(a.uout);
  for (int b = blockIdx.x; b < a.n_top + a.n_chains; b += gridDim.x) {
    const int4 d0 = *reinterpret_cast<const int4*>(a.seg + (long long)kSegInts * b);
    const int4 d1 = *reinterpret_cast<const int4*>(a.seg + (long long)kSegInts * b + 4);
    const int pb = d0.y, pl = d0.z, cb = d1.x, len = d1.y;
    if (!tree_active(a, d0.w, nu)) continue;  // a forest's tree that stopped keeps x and u
    const int L = pl + len;  // the path (root .. par), then the chain
    AT V = 0, U = 0;
    AT X = (act && tank && !lin) ? (AT)reinterpret_cast<const VT*>(a.p0)[(long long)d0.w * a.n_x + e] : (AT)0;
    for (int k0 = 0; k0 < L; k0 += KC) {
      const int q = min(KC, L - k0);
      __syncthreads();  // the previous chunk's node ids are consumed
      if (e < q) sid[e] = k0 + e < pl ? a.path_node[pb + k0 + e] : a.chain_node[cb + k0 + e - pl];
      __syncthreads();
      if (act) {
        for (int r = 0; r < q; ++r) {
          const long long m = sid[r];
          cp_async_elem(sh + r * n_k + e, H + m * n_k + e);
          if (HA) cp_async_elem(sa + r * n_k + e, HA + m * n_k + e);
          if (!lin) cp_async_elem(se + r * n_k + e, tank ? E + m * a.n_x + e : UH + m * a.n_u + i);
        }
        cp_async_wait_all();
      }
      if (a.A) {  // x_n = A x_parent + Bbar v_n + e_n (App. B): the state is shared per node
        const VT* Am = reinterpret_cast<const VT*>(a.A);
        for (int r = 0; r < q; ++r) {
          const int k = k0 + r;
          AT hv = 0, ev = 0;
          if (act) {
            hv = (AT)sh[r * n_k + e];
            if (HA) hv += (AT)sa[r * n_k + e];
            ev = lin ? (AT)0 : (AT)se[r * n_k + e];
          }
          __syncthreads();  // the previous node's reads of sX are done
          if (act && tank) sX[e] = X;
          __syncthreads();
          if (act) {
            if (tank) {
              AT ax = 0;
              for (int j = 0; j < a.n_x; ++j) ax += (AT)Am[(long long)e * a.n_x + j] * sX[j];
              V += hv;
              X = ax + V + ev;
            } else {
              U += hv;
            }
            if (k >= pl || (len == 0 && k == pl - 1)) {
              const long long m = sid[r];
              if (tank)
                XO[m * a.n_x + e] = (VT)X;
              else
                UO[m * a.n_u + i] = (VT)(U + ev);
            }
          }
        }
        continue;
      }
      if (!act) continue;
      for (int r = 0; r < q; ++r) {
        const int k = k0 + r;
        AT hv = (AT)sh[r * n_k + e];
        if (HA) hv += (AT)sa[r * n_k + e];
        const AT ev = lin ? (AT)0 : (AT)se[r * n_k + e];
        if (tank) {
          V += hv;
          X += V + ev;
        } else {
          U += hv;
        }
        // the segment's own nodes: the chain, or the top node that ends the path
        if (k >= pl || (len == 0 && k == pl - 1)) {
          const long long m = sid[r];
          if (tank)
            XO[m * a.n_x + e] = (VT)X;
          else
            UO[m * a.n_u + i] = (VT)(U + ev);
        }
      }
    }
  }
}

// Per-warp staging of prox_node (warp_prox_staged), 16-byte multiple.
template <typename VT>
__host__ __device__ size_t prox_stage_bytes(int n_x, int n_u) {
  const int n_k = n_x + n_u;
  return round_up((size_t)(2 * n_k + 2 * n_x) * 8 + (size_t)(2 * n_k + 2 * n_u) * sizeof(VT), 16);
}

// Phase P, node-parallel: one warp per node.  Dynamic shared memory: the barriers and
// vectors of carve (no pack slot), then kWarps staging regions (prox_stage_bytes).
template <typename VT, typename MT>
__global__ void __launch_bounds__(kThreads, 3) prox_node(const __grid_constant__ IterArgs a, int nu, int mode) {
  grid_dep_sync();
  using AT = typename Acc<MT>::T;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ AT bnd[5 * kThreads];  // x_s, x_max, x_min, u_max, u_min
  __shared__ unsigned long long ttab[3 * kTreeTable];
  Smem<MT> sm = carve<MT>(smem_raw, 0, a.n_x, a.n_u, a.n_v);
  // the forward sweep (when there is one) already took the stop decision
  const bool decide = !((mode & MODE_PROX) && nu >= 1);
  if (early_exit(a, nu, mode, sm.flag + 1, decide)) return;
  Kern<VT, MT> k(a, sm, 0, nu, mode);
  const bool do_prox = (mode & MODE_PROX) != 0 && nu >= 1;
  const bool do_bwd = (mode & (MODE_BWD | MODE_WONLY)) != 0;
  const int warp = threadIdx.x >> 5;
  if (do_prox && !k.linear()) {
    const int t = threadIdx.x;
    if (t < a.n_x) {
      bnd[t] = (AT)reinterpret_cast<const VT*>(a.x_s)[t];
      bnd[kThreads + t] = (AT)reinterpret_cast<const VT*>(a.x_max)[t];
      bnd[2 * kThreads + t] = (AT)reinterpret_cast<const VT*>(a.x_min)[t];
    }
    if (t < a.n_u) {
      bnd[3 * kThreads + t] = (AT)reinterpret_cast<const VT*>(a.u_max)[t];
      bnd[4 * kThreads + t] = (AT)reinterpret_cast<const VT*>(a.u_min)[t];
    }
    __syncthreads();
    unsigned char* stage = smem_raw + iter_smem_bytes<MT>(0, a.n_x, a.n_u, a.n_v) +
                           (size_t)warp * prox_stage_bytes<VT>(a.n_x, a.n_u);
    if (a.res_tree) {
      tree_table_clear(a, ttab);
      __syncthreads();
      k.ttab = ttab;
    }
    const int nn = a.node_list ? a.n_list : a.n;
    for (int j = blockIdx.x * kWarps + warp; j < nn; j += gridDim.x * kWarps) {
      const int m = a.node_list ? a.node_list[j] : j;
      const int r = a.res_tree ? a.tree_of[m] : -1;
      if (r >= 0 && !tree_active(a, r, nu)) continue;  // a forest's tree that stopped keeps its iterates
      k.warp_prox_staged(m, bnd, stage, r);
      __syncwarp();  // the lanes' reads of the staging are done before the next node's copies
    }
    if (a.res_tree) {
      __syncthreads();
      tree_table_flush(a, ttab, nu);
    }
  } else {
    const int nn = a.node_list ? a.n_list : a.n;
    for (int j = blockIdx.x * kWarps + warp; j < nn; j += gridDim.x * kWarps)
      k.warp_prox(a.node_list ? a.node_list[j] : j, do_prox, do_bwd && (!do_prox || k.linear()));
  }
  k.reduce_out(do_prox);
}

// Subtree sums out_n = in_n (+ beta_n) + sum over children c of out_c.  One CTA per chain
// (bottom-up in registers), then each top node is summed by the CTA whose arrival
// completes its children.  which = 0: s from xi = w[:, :n_x]; which = 1: r from g, in place.
// s of every node with a general A (App. B): s_n = xi_n + A' sum_{c in C(n)} s_c.  Along a
// chain the sum from below is multiplied by A' at every node, so the running vector is shared
// through shared memory and thread e forms entry e of A' s from column e of A (read through
// the cache; A is the same for every node).  Top nodes as in scan_kernel: the CTA whose
// arrival completes a node's children sums them and applies A'.
template <typename VT>
__device__ void scan_s_general_A(const IterArgs& a, int* flag) {
  __shared__ VT sv[kThreads];
  const int e = threadIdx.x, nx = a.n_x;
  const VT* in = reinterpret_cast<const VT*>(a.wbuf);
  VT* out = reinterpret_cast<VT*>(a.spub);
  const VT* A = reinterpret_cast<const VT*>(a.A);
  const long long is = a.n_k;
  // own + (A' sv)_e, once sv holds the vector to multiply (all threads call it)
  auto add_At = [&](VT own) {
    VT acc = own;
    if (e < nx)
      for (int j = 0; j < nx; ++j) acc += A[(long long)j * nx + e] * sv[j];
    return acc;
  };
  for (int ch = blockIdx.x; ch < a.n_chains; ch += gridDim.x) {
    const int cb = a.chain_off[ch], len = a.chain_off[ch + 1] - cb;
    int t = a.chain_parent[ch];
    VT cur = 0;  // s of the chain node below (none below the bottom leaf)
    for (int k = len - 1; k >= 0; --k) {
      const int m = a.chain_node[cb + k];
      const VT x = e < nx ? in[(long long)m * is + e] : (VT)0;
      __syncthreads();  // the previous node's reads of sv are done
      if (e < nx) sv[e] = cur;
      __syncthreads();
      cur = add_At(x);
      if (e < nx) out[(long long)m * nx + e] = cur;
    }
    while (t >= 0) {
      const int c0 = a.child_begin[t], cc = a.child_count[t], up = a.parent[t];
      const VT x = e < nx ? in[(long long)t * is + e] : (VT)0;
      __syncthreads();  // this CTA's outputs, then one fence, before its arrival
      if (e == 0) {
        fence_acq_rel_gpu();
        const int last = atomicAdd(&a.counters[t], 1) == cc - 1;
        if (last) {
          a.counters[t] = 0;
          fence_acq_rel_gpu();
        }
        flag[1] = last;
      }
      __syncthreads();
      if (!flag[1]) break;
      VT csum = 0;
      if (e < nx)
        for (int q = 0; q < cc; ++q) csum += ldcg(out + (long long)(c0 + q) * nx + e);
      if (e < nx) sv[e] = csum;
      __syncthreads();
      const VT v = add_At(x);
      if (e < nx) out[(long long)t * nx + e] = v;
      t = up;
    }
  }
}

template <typename VT>
__global__ void __launch_bounds__(kThreads) scan_kernel(const __grid_constant__ IterArgs a, int which, int nu,
                                                        int mode) {
  grid_dep_sync();
  __shared__ int flag[2];
  if (early_exit(a, nu, mode, flag, false)) return;
  const int e = threadIdx.x;
  const int W = which == 0 ? a.n_x : a.n_v;
  const bool with_beta = which == 1 && (mode & (MODE_LINEAR | MODE_DELTA)) == 0;
  const VT* in = reinterpret_cast<const VT*>(which == 0 ? a.wbuf : a.rpub);
  VT* out = reinterpret_cast<VT*>(which == 0 ? a.spub : a.rpub);
  const VT* beta = reinterpret_cast<const VT*>(a.beta);
  const long long is = which == 0 ? a.n_k : a.n_v, os = W;
  constexpr int B = 32;  // chain nodes whose loads are in flight together
  constexpr int C = 8;   // children of a top node loaded together
  if (which == 0 && a.A) {
    scan_s_general_A<VT>(a, flag);
    return;
  }
  for (int ch = blockIdx.x; ch < a.n_chains; ch += gridDim.x) {
    const int cb = a.chain_off[ch], len = a.chain_off[ch + 1] - cb;
    int t = a.chain_parent[ch];
    if (e < W) {
      VT acc = 0;
      for (int k1 = len; k1 > 0; k1 -= B) {  // nodes k1-1 .. k1-B, bottom-up: ids, then vectors, then sums
        int id[B];
        VT v[B];
#pragma unroll
        for (int j = 0; j < B; ++j) id[j] = k1 - 1 - j >= 0 ? a.chain_node[cb + k1 - 1 - j] : -1;
#pragma unroll
        for (int j = 0; j < B; ++j) {
          v[j] = 0;
          if (id[j] >= 0) {
            v[j] = in[(long long)id[j] * is + e];
            if (with_beta) v[j] += beta[(long long)id[j] * a.n_v + e];
          }
        }
#pragma unroll
        for (int j = 0; j < B; ++j) {
          if (id[j] >= 0) {
            acc += v[j];
            out[(long long)id[j] * os + e] = acc;
          }
        }
      }
    }
    while (t >= 0) {
      // the top node's own term and its children's range are loaded before the arrival
      // (only the last arriving CTA uses them, and only it writes out[t], after every
      // arrival); the children's sums, written by other CTAs, after it
      const int c0 = a.child_begin[t], cc = a.child_count[t], up = a.parent[t];
      VT v = 0;
      if (e < W) {
        v = in[(long long)t * is + e];
        if (with_beta) v += beta[(long long)t * a.n_v + e];
      }
      __syncthreads();  // this CTA's outputs, then one fence, before its arrival (as in arrive)
      if (e == 0) {
        fence_acq_rel_gpu();
        const int last = atomicAdd(&a.counters[t], 1) == cc - 1;
        if (last) {
          a.counters[t] = 0;
          fence_acq_rel_gpu();
        }
        flag[1] = last;
      }
      __syncthreads();
      if (!flag[1]) break;
      if (e < W) {
        for (int q = 0; q < cc; q += C) {
          VT cv8[C];
#pragma unroll
          for (int j = 0; j < C; ++j) cv8[j] = q + j < cc ? ldcg(out + (long long)(c0 + q + j) * os + e) : (VT)0;
#pragma unroll
          for (int j = 0; j < C; ++j)
            if (q + j < cc) v += cv8[j];
        }
        out[(long long)t * os + e] = v;
      }
      t = up;
    }
  }
}

// Per-node mat-vec launches: CTA b handles nodes b, b + G, ... and streams their packs
// through S shared-memory slots with cp.async.bulk, so that the copies of the next
// nodes overlap the current node's mat-vecs.  gt: g_n = [Bbar; L]_n' [s_n; psi_n];
// dh: delta = Lambda_n r_n / (2 p_n), h_n = [Bbar; L]_n delta.
template <typename VT, typename MT, bool DH>
__global__ void __launch_bounds__(kThreads, 1) node_mv(const __grid_constant__ IterArgs a, int S, int nu, int mode) {
  grid_dep_sync();
  using AT = typename Acc<MT>::T;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Smem<MT> sm = carve<MT>(smem_raw, S, a.n_x, a.n_u, a.n_v, DH);
  if (early_exit(a, nu, mode, sm.flag + 1, false)) return;
  const int tid = threadIdx.x;
  const MT* packs = reinterpret_cast<const MT*>(a.packs);
  const long long kp = kpad<MT>(a.n_k, a.n_v);
  const uint32_t kb = (uint32_t)sm.kbytes, lb = (uint32_t)sm.lbytes;
  const int G = gridDim.x;
  const int count = a.n > (int)blockIdx.x ? (a.n - 1 - (int)blockIdx.x) / G + 1 : 0;
  if (tid == 0) {
    for (int q = 0; q < S; ++q) mbar_init(&sm.barK[q], 1);
    fence_barrier_init();
  }
  for (int j = a.n_v + tid; j < sm.ld; j += kThreads) sm.dv[j] = 0;
  __syncthreads();
  // shared pack (pack_stride 0): one copy into slot 0, kept for every node
  const bool shared = a.pack_stride == 0;
  if (shared) S = 1;
  auto issue = [&](int q) {  // thread 0: copies of the q-th node into slot q % S
    const int m = blockIdx.x + q * G;
    const int slot = q % S;
    fence_proxy_async();
    mbar_expect_tx(&sm.barK[slot], kb + (DH ? lb : 0u));
    const unsigned char* src = reinterpret_cast<const unsigned char*>(packs + (long long)m * a.pack_stride);
    bulk_g2s(sm.K(slot), src, kb, &sm.barK[slot]);
    if (DH) bulk_g2s(sm.Lm(slot), src + kp * sizeof(MT), lb, &sm.barK[slot]);
  };
  if (tid == 0)
    for (int q = 0; q < S && q < count && (!shared || q == 0); ++q) issue(q);
  const VT* wb = reinterpret_cast<const VT*>(a.wbuf);
  const VT* sp = reinterpret_cast<const VT*>(a.spub);
  VT* rp = reinterpret_cast<VT*>(a.rpub);
  int failed_at = -1;
  for (int q = 0; q < count; ++q) {
    const long long m = blockIdx.x + (long long)q * G;
    const int slot = q % S;
    // node vectors into shared memory while the copy lands
    if (DH) {
      if (tid < a.n_v) sm.rv[tid] = (AT)rp[m * a.n_v + tid];
    } else if (tid < a.n_k) {
      sm.yv[tid] = tid < a.n_x ? (AT)sp[m * a.n_x + tid] : (AT)wb[m * a.n_k + tid];
    }
    const bool ok = (shared && q > 0) || mbar_wait(&sm.barK[slot], shared ? 0 : (q / S) & 1, a.wait_ns);
    if (__syncthreads_or(!ok)) {
      failed_at = q;
      break;
    }
    if (DH) {
      matvec_t<MT, AT>(sm.Lm(slot), a.n_v, a.n_v, sm.ld, sm.rv, sm.dv, sm.part);  // Lambda is symmetric
      if (a.pscale) {  // shared pack: delta = (Lambda r) / (2 p_n)
        const AT sc = (AT)reinterpret_cast<const VT*>(a.pscale)[m];
        if (tid < a.n_v) sm.dv[tid] *= sc;
        __syncthreads();
      }
      matvec_n<MT, AT>(sm.K(slot), a.n_k, sm.ld, sm.dv, sm.yv);
      if (tid < a.n_k) {
        VT* h = reinterpret_cast<VT*>(a.h);
        if (mode & MODE_ANCHOR) {
          reinterpret_cast<VT*>(a.ha)[m * a.n_k + tid] = (VT)sm.yv[tid];
          h[m * a.n_k + tid] = (VT)0;
        } else {
          h[m * a.n_k + tid] = (VT)sm.yv[tid];
        }
      }
    } else {
      matvec_t<MT, AT>(sm.K(slot), a.n_k, a.n_v, sm.ld, sm.yv, sm.gv, sm.part);
      if (tid < a.n_v) rp[m * a.n_v + tid] = (VT)sm.gv[tid];
    }
    __syncthreads();  // the slot and the vectors are free again
    if (tid == 0 && !shared && q + S < count) issue(q + S);
  }
  if (failed_at >= 0 && tid == 0) {
    // let this CTA's copies still in flight (nodes failed_at .. failed_at + S - 1) land,
    // each wait bounded, before leaving
    a.flags[1] = SMPC_ETIMEOUT;
    const int end = shared ? min(count, 1) : min(count, failed_at + S);
    for (int q = failed_at; q < end; ++q) mbar_wait(&sm.barK[q % S], (q / S) & 1);
  }
}

// ------------------------------------------------------------------ shards
// Cut parent j (a top node with chain children): the sums over this GPU's chain heads
// below it of s (n_x entries) and r (n_v entries); one CTA per cut parent.
template <typename VT>
__global__ void cut_sums_kernel(IterArgs a, int n_cut, const int* cut_off, const int* cut_heads, VT* out) {
  const int W = a.n_x + a.n_v;
  const VT* sp = reinterpret_cast<const VT*>(a.spub);
  const VT* rp = reinterpret_cast<const VT*>(a.rpub);
  for (int j = blockIdx.x; j < n_cut; j += gridDim.x) {
    for (int e = threadIdx.x; e < W; e += blockDim.x) {
      VT v = 0;
      for (int q = cut_off[j]; q < cut_off[j + 1]; ++q) {  // heads in index order
        const long long h = cut_heads[q];
        v += e < a.n_x ? sp[h * a.n_x + e] : rp[h * a.n_v + (e - a.n_x)];
      }
      out[(long long)j * W + e] = v;
    }
  }
}
// The exchanged totals into the chain children of each cut parent: the first chain child
// carries the total, the others zero, so that the top pass's sum over children is the
// sum over every GPU's chains.
template <typename VT>
__global__ void cut_scatter_kernel(IterArgs a, int n_cut, const int* chl_off, const int* chl, const VT* in) {
  const int W = a.n_x + a.n_v;
  VT* sp = reinterpret_cast<VT*>(a.spub);
  VT* rp = reinterpret_cast<VT*>(a.rpub);
  for (int j = blockIdx.x; j < n_cut; j += gridDim.x) {
    for (int q = chl_off[j]; q < chl_off[j + 1]; ++q) {
      const long long c = chl[q];
      const bool first = q == chl_off[j];
      for (int e = threadIdx.x; e < W; e += blockDim.x) {
        const VT v = first ? in[(long long)j * W + e] : (VT)0;
        if (e < a.n_x)
          sp[c * a.n_x + e] = v;
        else
          rp[c * a.n_v + (e - a.n_x)] = v;
      }
    }
  }
}

// ------------------------------------------------------------------ helpers
template <typename VT, typename MT>
__global__ void pack_kernel(int n, int n_k, int n_v, const double* K, const double* Lam, const double* prob,
                            MT* packs, long long stride) {
  const long long kp = kpad<MT>(n_k, n_v), lp = lpad<MT>(n_v);
  const int ld = row_stride<MT>(n_v);
  for (int m = blockIdx.x; m < n; m += gridDim.x) {
    MT* dst = packs + (long long)m * stride;
    const double inv = prob ? 1.0 / (2.0 * prob[m]) : 1.0;  // no prob: the shared pack, Lambda unscaled
    for (long long q = threadIdx.x; q < kp; q += blockDim.x) {
      const long long i = q / ld, j = q % ld;
      dst[q] = (MT)(i < n_k && j < n_v ? K[i * n_v + j] : 0.0);
    }
    for (long long q = threadIdx.x; q < lp; q += blockDim.x) {
      const long long i = q / ld, j = q % ld;
      dst[kp + q] = (MT)(i < n_v && j < n_v ? Lam[i * n_v + j] * inv : 0.0);
    }
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
      D -= pm * (par >= 0 ? a.uhat64[(long long)par * a.n_u + i] : a.q[(long long)a.tree_of[m] * a.n_u + i]);
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
  using ST = typename St<VT>::T;
  __shared__ int it;
  if (threadIdx.x == 0) {
    it = a.flags[0];
    if (it < 0) it = max_iters;
  }
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0) a.flags[0] = it;
  if (!dst) return;
  const int nd = 2 * a.n_x + a.n_u;
  const long long total = (long long)a.n * nd;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    int itn = it;  // a forest's tree that stopped early ends at its own iteration count
    if (a.tree_done) {
      const int d = a.tree_done[a.tree_of[i / nd]];
      if (d >= 0) itn = d;
    }
    const ST* src = reinterpret_cast<const ST*>((itn & 1) ? a.ybuf1 : a.ybuf0);
    dst[i] = (VT)st_val(src[i]);
  }
}

template <typename VT>
__global__ void init_duals_kernel(IterArgs a, int warm) {
  // cold: y^0 = y^{-1} = 0 ; warm: both = the final dual of the previous solve
  using ST = typename St<VT>::T;
  const int nd = 2 * a.n_x + a.n_u;
  const long long total = (long long)a.n * nd;
  const int it = a.flags[0];
  ST* y0 = reinterpret_cast<ST*>(a.ybuf0);
  ST* y1 = reinterpret_cast<ST*>(a.ybuf1);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    ST v = st_from<ST>(0.0);
    if (warm) {  // each tree of a forest ended at its own iteration count
      int itn = it;
      if (a.tree_done) {
        const int d = a.tree_done[a.tree_of[i / nd]];
        if (d >= 0) itn = d;
      }
      v = ((itn & 1) ? y1 : y0)[i];
    }
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

// Shared pack (pack_stride 0): the pack is copied into shared memory once per CTA and
// applied to kNB nodes per pass, so that each 16-byte matrix load feeds kNB nodes.
//   gt: g_b = [Bbar; L]' y_b,  y_b = [s_b; psi_b]
//   dh: delta_b = (Lambda r_b) / (2 p_b),  h_b = [Bbar; L] delta_b
// The transposed products use the column-group layout of matvec_t (thread (g, p): the
// V columns of group g over row slice p, slices added in a fixed order); [Bbar; L] delta
// gives each thread one row and all kNB dot products.
constexpr int kNB = 8;

template <typename MT>
__host__ __device__ inline int multi_slices(int n_v) {
  const int ld = row_stride<MT>(n_v);
  const int G = ld / (16 / (int)sizeof(MT));
  int P = kThreads / G;
  return P > 16 ? 16 : P;
}
template <typename MT>
__host__ __device__ inline size_t multi_smem_bytes(int n_x, int n_u, int n_v, bool dh) {
  using AT = typename Acc<MT>::T;
  const int n_k = n_x + n_u, ld = row_stride<MT>(n_v);
  size_t b = round_up((long long)kpad<MT>(n_k, n_v) * sizeof(MT), 16);
  if (dh) b += round_up((long long)lpad<MT>(n_v) * sizeof(MT), 16);
  b += 16;                                                          // mbarrier
  const size_t ldk = round_up(n_k, 4);
  b += (size_t)kNB * ((ldk > (size_t)ld ? ldk : (size_t)ld) + ld) * sizeof(AT);  // inputs, outputs
  b += (size_t)multi_slices<MT>(n_v) * kNB * ld * sizeof(AT);       // slice partial sums
  return round_up(b, 128);
}

// out[b][j] = sum_i A[i*ld + j] x[b][i] (i < R, j < C) for kNB vectors x[b] (stride xs)
template <typename MT, typename AT>
__device__ void multi_t(const MT* A, int R, int C, int ld, const AT* x, int xs, AT* out, int os, AT* part) {
  constexpr int V = Vec<MT>::V;
  const int t = threadIdx.x;
  const int G = ld / V;
  const int P = multi_slices<MT>(C);
  const int rc = (R + P - 1) / P;
  if (t < P * G) {
    const int g = t % G, p = t / G;
    const int i0 = p * rc, i1 = min(R, i0 + rc);
    AT acc[kNB][V];
#pragma unroll
    for (int b = 0; b < kNB; ++b)
#pragma unroll
      for (int k = 0; k < V; ++k) acc[b][k] = 0;
    const MT* col = A + g * V;
#pragma unroll 2
    for (int i = i0; i < i1; ++i) {
      AT av[V];
      ld16(col + (long long)i * ld, av);
#pragma unroll
      for (int b = 0; b < kNB; ++b) {
        const AT xb = x[b * xs + i];
#pragma unroll
        for (int k = 0; k < V; ++k) acc[b][k] += av[k] * xb;
      }
    }
#pragma unroll
    for (int b = 0; b < kNB; ++b) {
      AT* dst = part + ((long long)p * kNB + b) * ld + g * V;
#pragma unroll
      for (int k = 0; k < V; ++k) dst[k] = acc[b][k];
    }
  }
  __syncthreads();
  for (int q = t; q < kNB * C; q += kThreads) {
    const int b = q / C, j = q % C;
    AT s = 0;
    for (int p = 0; p < P; ++p) s += part[((long long)p * kNB + b) * ld + j];  // fixed order
    out[b * os + j] = s;
  }
  __syncthreads();
}

template <typename VT, typename MT, bool DH>
__global__ void __launch_bounds__(kThreads, 1) node_mv_shared(const __grid_constant__ IterArgs a, int nu, int mode) {
  grid_dep_sync();
  using AT = typename Acc<MT>::T;
  constexpr int V = Vec<MT>::V;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int flag[2];
  if (early_exit(a, nu, mode, flag, false)) return;
  const int tid = threadIdx.x;
  const int n_k = a.n_k, n_v = a.n_v, ld = row_stride<MT>(n_v);
  const size_t kb = (size_t)kpad<MT>(n_k, n_v) * sizeof(MT), lb = (size_t)lpad<MT>(n_v) * sizeof(MT);
  unsigned char* p = smem_raw;
  const MT* K = reinterpret_cast<const MT*>(p);
  p += round_up((long long)kb, 16);
  const MT* Lm = reinterpret_cast<const MT*>(p);
  if (DH) p += round_up((long long)lb, 16);
  uint64_t* bar = reinterpret_cast<uint64_t*>(p);
  p += 16;
  const int ldk = (int)round_up(n_k, 4);
  const int lx = ldk > ld ? ldk : ld;
  AT* xin = reinterpret_cast<AT*>(p);  // GT: y (kNB x ldk); DH: r (kNB x ld)
  AT* dv = xin + kNB * lx;             // GT: g; DH: delta (kNB x ld, zero beyond n_v)
  p += (size_t)kNB * (lx + ld) * sizeof(AT);
  AT* part = reinterpret_cast<AT*>(p);
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
    fence_proxy_async();
    const unsigned char* src = reinterpret_cast<const unsigned char*>(a.packs);
    mbar_expect_tx(bar, (uint32_t)(kb + (DH ? lb : 0)));
    bulk_g2s(const_cast<MT*>(K), src, (uint32_t)kb, bar);
    if (DH) bulk_g2s(const_cast<MT*>(Lm), src + kpad<MT>(n_k, n_v) * sizeof(MT), (uint32_t)lb, bar);
  }
  for (int q = tid; q < kNB * ld; q += kThreads) dv[q] = 0;
  __syncthreads();
  const bool ok = mbar_wait(bar, 0);
  if (__syncthreads_or(!ok)) {
    if (tid == 0) {
      a.flags[1] = SMPC_ETIMEOUT;
      mbar_wait(bar, 0);  // bounded: let the copy in flight land before leaving
    }
    return;
  }
  const VT* wb = reinterpret_cast<const VT*>(a.wbuf);
  const VT* sp = reinterpret_cast<const VT*>(a.spub);
  VT* rp = reinterpret_cast<VT*>(a.rpub);
  const VT* ps = reinterpret_cast<const VT*>(a.pscale);
  const int batches = (a.n + kNB - 1) / kNB;
  for (int bt = blockIdx.x; bt < batches; bt += gridDim.x) {
    const long long m0 = (long long)bt * kNB;
    const int nb = min(kNB, a.n - (int)m0);  // nodes of this batch; the others read zeros
    if (!DH) {
      for (int q = tid; q < kNB * n_k; q += kThreads) {
        const int b = q / n_k, i = q % n_k;
        AT v = 0;
        if (b < nb) v = i < a.n_x ? (AT)sp[(m0 + b) * a.n_x + i] : (AT)wb[(m0 + b) * n_k + i];
        xin[b * ldk + i] = v;
      }
      __syncthreads();
      multi_t<MT, AT>(K, n_k, n_v, ld, xin, ldk, dv, ld, part);
      for (int q = tid; q < nb * n_v; q += kThreads) {
        const int b = q / n_v, j = q % n_v;
        rp[(m0 + b) * n_v + j] = (VT)dv[b * ld + j];
      }
      __syncthreads();
    } else {
      for (int q = tid; q < kNB * n_v; q += kThreads) {
        const int b = q / n_v, j = q % n_v;
        xin[b * ld + j] = b < nb ? (AT)rp[(m0 + b) * n_v + j] : (AT)0;
      }
      __syncthreads();
      multi_t<MT, AT>(Lm, n_v, n_v, ld, xin, ld, dv, ld, part);  // Lambda is symmetric
      for (int q = tid; q < kNB * n_v; q += kThreads) {
        const int b = q / n_v, j = q % n_v;
        dv[b * ld + j] *= b < nb ? (AT)ps[m0 + b] : (AT)0;
      }
      __syncthreads();
      // h_b[i] = [Bbar; L]_i . delta_b: thread i, all kNB nodes per row chunk
      if (tid < n_k) {
        AT acc[kNB];
#pragma unroll
        for (int b = 0; b < kNB; ++b) acc[b] = 0;
        const MT* row = K + (long long)tid * ld;
        for (int g = 0; g < ld / V; ++g) {
          AT av[V];
          ld16(row + g * V, av);
#pragma unroll
          for (int b = 0; b < kNB; ++b) {
            AT dvv[V];
            ldx(dv + b * ld + g * V, dvv);
#pragma unroll
            for (int k = 0; k < V; ++k) acc[b] += av[k] * dvv[k];
          }
        }
        VT* h = reinterpret_cast<VT*>(a.h);
        VT* ha = reinterpret_cast<VT*>(a.ha);
#pragma unroll
        for (int b = 0; b < kNB; ++b) {
          if (b >= nb) continue;
          const long long q = (m0 + b) * n_k + tid;
          if (mode & MODE_ANCHOR) {
            ha[q] = (VT)acc[b];
            h[q] = (VT)0;
          } else {
            h[q] = (VT)acc[b];
          }
        }
      }
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------------ tensor-core Lambda / [Bbar; L]
// bfloat16 shared pack, anchored (delta) launches: for tn nodes at a time (16, 32 or 64) the
// two products are dense GEMMs on the 5th-generation tensor cores,
//   D1 = Lambda_pad (128 x Kp) . R (Kp x tn),   delta = D1 / (2 p_b) rounded to bfloat16,
//   D2 = [Bbar; L]_pad (256 x Kp) . delta (Kp x tn)  (two 128-row tiles),
// Kp = n_v rounded up to 16.  Operands sit in shared memory K-major without swizzle, in
// 8-row x 16-byte core matrices; accumulators (float32) sit in tensor memory.  One thread
// issues the MMAs and commits them to an mbarrier; every wait is bounded.  The vectors
// are rounded to bfloat16 here: in a delta launch they are the changes since the anchor,
// whose rounding is an error proportional to |w - w_a| (the anchors run in float32).
constexpr int kTcMaxN = 64;     // nodes per GEMM (the N of the MMA): 16, 32 or 64
constexpr int kTcCore = 128;    // bytes per core matrix
// threads of a tensor-core CTA: eight warps share the vector work (conversions, layout
// scatters, result write-back); warp w reads tensor-memory lanes 32 (w mod 4) .. + 31 (the
// quarter a warp may access) and the 16-column chunks c0 = 16 (w div 4), + 32, ...
constexpr int kTcThreads = 256;

__host__ __device__ inline int tc_kp(int n_v) { return (n_v + 15) / 16 * 16; }
// float32 R block of one batch (tn nodes' r, contiguous in rpub), staged by a bulk copy
__host__ __device__ inline size_t tc_stage_bytes(int n_v, int tn) { return (size_t)tn * n_v * sizeof(float); }
__host__ __device__ inline size_t tc_smem_bytes(int n_v, int tn) {
  const size_t sbo = (size_t)tc_kp(n_v) / 8 * kTcCore;  // bytes per 8-row group
  return (128 / 8) * sbo + (256 / 8) * sbo + 2 * (size_t)(tn / 8) * sbo + 64 + 2 * tc_stage_bytes(n_v, tn);
}
__host__ __device__ inline bool tc_fits(int n_x, int n_u, int n_v) { return n_v <= 128 && n_x + n_u <= 256; }

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version; base offset 0, no swizzle
  return d;
}
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
               " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
               "l"(da), "l"(db), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t addr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tc_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// byte offset of element (row r, k) of a K-major operand in core-matrix layout
__device__ __forceinline__ int tc_off(int r, int k, int sbo) {
  return (r >> 3) * sbo + (k >> 3) * kTcCore + (r & 7) * 16 + (k & 7) * 2;
}

template <typename VT>
__global__ void __launch_bounds__(kTcThreads, 1) node_mv_tc(const __grid_constant__ IterArgs a, int tn, int nu, int mode) {
  grid_dep_sync();
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ int flag[2];
  if (early_exit(a, nu, mode, flag, false)) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int qw = warp & 3, hc = warp >> 2;  // tensor-memory lane quarter, column-chunk parity
  const int n_k = a.n_k, n_v = a.n_v, Kp = tc_kp(n_v), ld = row_stride<__nv_bfloat16>(n_v);
  const int sbo = Kp / 8 * kTcCore;
  unsigned char* A1 = smem_raw;                   // Lambda, 128 rows
  unsigned char* A2 = A1 + 16 * sbo;              // [Bbar; L], 256 rows
  unsigned char* B1 = A2 + 32 * sbo;              // R (tn rows)
  unsigned char* B2 = B1 + (tn / 8) * sbo;        // delta (tn rows)
  uint64_t* bar = reinterpret_cast<uint64_t*>(B2 + (tn / 8) * sbo);  // MMA completion
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  uint64_t* sbar = bar + 2;  // the two R staging buffers' copies
  // R of a whole batch is tn consecutive rows of rpub (tn n_v floats, a 16-byte multiple at a
  // 16-byte aligned offset): one bulk copy per batch, issued one batch ahead into the other
  // buffer, so that a batch's R is on chip when its MMAs are due (the last batch of a tree
  // with fewer than tn nodes left reads its rows with plain loads)
  const uint32_t sbytes = (uint32_t)tc_stage_bytes(n_v, tn);
  unsigned char* stage0 = B2 + (tn / 8) * sbo + 64;  // buffer sb at stage0 + sb * sbytes
  // pack -> core-matrix layout, zero padding (16-byte chunks; the pack's rows are ld >= n_v wide)
  const __nv_bfloat16* pk = reinterpret_cast<const __nv_bfloat16*>(a.packs);
  const long long kp = kpad<__nv_bfloat16>(n_k, n_v);
  const int kc = Kp / 8;
  for (int q = tid; q < (128 + 256) * kc; q += blockDim.x) {
    const int row = q / kc, c = q % kc;
    uint4 v = make_uint4(0, 0, 0, 0);
    unsigned char* dst;
    if (row < 128) {
      if (row < n_v && 8 * c < ld) v = *reinterpret_cast<const uint4*>(pk + kp + (long long)row * ld + 8 * c);
      dst = A1 + tc_off(row, 8 * c, sbo);
    } else {
      const int r = row - 128;
      if (r < n_k && 8 * c < ld) v = *reinterpret_cast<const uint4*>(pk + (long long)r * ld + 8 * c);
      dst = A2 + tc_off(r, 8 * c, sbo);
    }
    *reinterpret_cast<uint4*>(dst) = v;
  }
  for (int q = tid; q < 2 * (tn / 8) * sbo / 16; q += blockDim.x)
    reinterpret_cast<uint4*>(B1)[q] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init(&sbar[0], 1);
    mbar_init(&sbar[1], 1);
    fence_barrier_init();
  }
  if (warp == 0) {  // 3 tn accumulator columns: D1, D2 rows 0-127, D2 rows 128-255 (tn <= 64)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)), "r"(256));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_proxy_async();
  tc_sync();
  const uint32_t tmem = *tslot;
  const uint32_t d1 = tmem, d2a = tmem + tn, d2b = tmem + 2 * tn;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(tn >> 3) << 17) | (8u << 24);
  const VT* rp = reinterpret_cast<const VT*>(a.rpub);
  const VT* ps = reinterpret_cast<const VT*>(a.pscale);
  VT* h = reinterpret_cast<VT*>(a.h);
  uint32_t phase = 0;
  bool failed = false;
  const int batches = (a.n + tn - 1) / tn;
  auto full = [&](int bt) { return bt < batches && (long long)(bt + 1) * tn <= a.n; };
  uint32_t sphase = 0;   // bit sb: the phase of buffer sb's barrier to wait for
  uint32_t pending = 0;  // bit sb: a copy into buffer sb issued and not yet awaited
  auto stage_copy = [&](int bt, int sb) {
    if (tid == 0) {
      fence_proxy_async();  // the buffer's last reads (generic) before the copy's writes (async)
      mbar_expect_tx(&sbar[sb], sbytes);
      bulk_g2s(stage0 + (size_t)sb * sbytes, rp + (long long)bt * tn * n_v, sbytes, &sbar[sb]);
    }
    pending |= 1u << sb;
  };
  if (full(blockIdx.x)) stage_copy(blockIdx.x, 0);
  int it = 0;
  for (int bt = blockIdx.x; bt < batches && !failed; bt += gridDim.x, ++it) {
    const long long m0 = (long long)bt * tn;
    const int nb = min(tn, a.n - (int)m0);
    const int sb = it & 1;
    const bool staged = full(bt);
    // the next batch's R into the other buffer, whose last reads ended at the previous batch's barriers
    if (full(bt + (int)gridDim.x)) stage_copy(bt + (int)gridDim.x, sb ^ 1);
    if (staged) {
      if (mbar_wait(&sbar[sb], (sphase >> sb) & 1u)) {
        sphase ^= 1u << sb;
        pending &= ~(1u << sb);
      } else {
        failed = true;
      }
      if (__syncthreads_or(failed)) {
        failed = true;
        break;
      }
    }
    // R: row b = node m0 + b, bfloat16
    const float* sr = reinterpret_cast<const float*>(stage0 + (size_t)sb * sbytes);
    for (int q = tid; q < tn * n_v; q += blockDim.x) {
      const int b = q / n_v, j = q % n_v;
      const float v = staged ? sr[q] : (b < nb ? (float)rp[(m0 + b) * n_v + j] : 0.f);
      *reinterpret_cast<__nv_bfloat16*>(B1 + tc_off(b, j, sbo)) = __float2bfloat16_rn(v);
    }
    fence_proxy_async();
    tc_sync();
    if (tid == 0) {
      for (int ks = 0; ks < Kp / 16; ++ks)
        umma_bf16(d1, umma_desc(smem_u32(A1) + ks * 2 * kTcCore, kTcCore, sbo),
                  umma_desc(smem_u32(B1) + ks * 2 * kTcCore, kTcCore, sbo), idesc, ks > 0);
      umma_commit(bar);
    }
    if (!mbar_wait(bar, phase)) failed = true;
    phase ^= 1;
    if (__syncthreads_or(failed)) {
      failed = true;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // delta = D1 / (2 p_b): warp w reads rows 32 (w mod 4) .. + 31 (the entries of delta)
    {
      const int i = 32 * qw + lane;
      for (int c0 = 16 * hc; c0 < tn; c0 += 32) {
        float v[16];
        tmem_ld16(d1 + ((uint32_t)(32 * qw) << 16) + c0, v);
        if (i < Kp) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int b = c0 + j;
            const float sc = (b < nb && i < n_v) ? (float)ps[m0 + b] : 0.f;
            *reinterpret_cast<__nv_bfloat16*>(B2 + tc_off(b, i, sbo)) = __float2bfloat16_rn(v[j] * sc);
          }
        }
      }
    }
    fence_proxy_async();
    tc_sync();
    if (tid == 0) {
      for (int t = 0; t < 2; ++t)
        for (int ks = 0; ks < Kp / 16; ++ks)
          umma_bf16(t ? d2b : d2a, umma_desc(smem_u32(A2) + t * 16 * sbo + ks * 2 * kTcCore, kTcCore, sbo),
                    umma_desc(smem_u32(B2) + ks * 2 * kTcCore, kTcCore, sbo), idesc, ks > 0);
      umma_commit(bar);
    }
    if (!mbar_wait(bar, phase)) failed = true;
    phase ^= 1;
    if (__syncthreads_or(failed)) {
      failed = true;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    for (int t = 0; t < 2; ++t) {
      const int i = 128 * t + 32 * qw + lane;  // row of [Bbar; L], entry of h
      for (int c0 = 16 * hc; c0 < tn; c0 += 32) {
        float v[16];
        tmem_ld16((t ? d2b : d2a) + ((uint32_t)(32 * qw) << 16) + c0, v);
        if (i < n_k) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (c0 + j < nb) h[(m0 + c0 + j) * n_k + i] = (VT)v[j];
        }
      }
    }
    tc_sync();  // B1, B2 and the accumulators are free for the next batch
  }
  if (failed && tid == 0) {
    a.flags[1] = SMPC_ETIMEOUT;
    mbar_wait(bar, phase ^ 1);  // bounded: let the MMAs in flight finish before freeing tensor memory
  }
  if (failed)  // bounded: let the staging copies in flight land before the CTA's shared memory goes
    for (int sb = 0; sb < 2; ++sb)
      if ((pending >> sb) & 1u) mbar_wait(&sbar[sb], (sphase >> sb) & 1u);
  tc_sync();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
}

// [Bbar; L]' y of the delta launches of a bfloat16 shared pack (the node-parallel schedule's
// second launch) as GEMMs on the tensor cores, tn nodes at a time:
//   D = Kt_pad (128 x Kq) . Y (Kq x tn),   Kt = [Bbar; L]' (n_v x n_k),  Kq = n_k rounded up to 16,
// y_b = [s_b; psi_b] (the subtree sum s from the scan, psi from w) rounded to bfloat16 - in a
// delta launch they are changes since the anchor, as in node_mv_tc - and g_b = D[:, b] to
// rpub, where the scan of r adds beta and the children.  Kt is built once per CTA by
// transposing the pack's rows in shared memory.  A batch's s and w rows (contiguous, 16-byte
// multiples at 16-byte aligned offsets) arrive by two bulk copies issued one batch ahead into
// the other of two staging buffers.  Every wait is bounded.
__host__ __device__ inline int tc_kq(int n_k) { return (n_k + 15) / 16 * 16; }
__host__ __device__ inline size_t gt_stage_bytes(int n_x, int n_k, int tn) {
  return (size_t)tn * (n_x + n_k) * sizeof(float);
}
__host__ __device__ inline size_t gt_smem_bytes(int n_x, int n_k, int tn) {
  const size_t sbo = (size_t)tc_kq(n_k) / 8 * kTcCore;  // bytes per 8-row group
  return (128 / 8) * sbo + (size_t)(tn / 8) * sbo + 64 + 2 * gt_stage_bytes(n_x, n_k, tn);
}
// element t (0..7) of the 8 bfloat16 values in v, as its 16 bits
__device__ __forceinline__ unsigned short bf16_bits(const uint4& v, int t) {
  const uint32_t w = t < 2 ? v.x : t < 4 ? v.y : t < 6 ? v.z : v.w;
  return (unsigned short)((t & 1) ? (w >> 16) : (w & 0xffffu));
}

template <typename VT>
__global__ void __launch_bounds__(kTcThreads, 1) node_gt_tc(const __grid_constant__ IterArgs a, int tn, int nu, int mode) {
  grid_dep_sync();
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ int flag[2];
  if (early_exit(a, nu, mode, flag, false)) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int qw = warp & 3, hc = warp >> 2;  // tensor-memory lane quarter, column-chunk parity
  const int n_x = a.n_x, n_k = a.n_k, n_v = a.n_v, Kq = tc_kq(n_k), ld = row_stride<__nv_bfloat16>(n_v);
  const int sbo = Kq / 8 * kTcCore;
  unsigned char* At = smem_raw;                                    // Kt: 128 rows (n_v used), Kq columns
  unsigned char* Bm = At + 16 * sbo;                               // Y: tn rows
  uint64_t* bar = reinterpret_cast<uint64_t*>(Bm + (tn / 8) * sbo);  // MMA completion
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  uint64_t* sbar = bar + 2;                                        // the two staging buffers' copies
  const uint32_t sx = (uint32_t)((size_t)tn * n_x * sizeof(float));  // s rows, then w rows
  const uint32_t sbytes = (uint32_t)gt_stage_bytes(n_x, n_k, tn);
  unsigned char* stage0 = Bm + (tn / 8) * sbo + 64;               // buffer sb at stage0 + sb * sbytes
  for (int q = tid; q < (16 + tn / 8) * sbo / 16; q += blockDim.x) reinterpret_cast<uint4*>(At)[q] = make_uint4(0, 0, 0, 0);
  __syncthreads();  // zero padding (rows n_v .. 127, columns n_k .. Kq - 1) before the scattered writes
  // Kt[j][i] = [Bbar; L][i][j]: 16-byte chunks of the pack's rows, each spread over 8 rows of Kt
  const __nv_bfloat16* pk = reinterpret_cast<const __nv_bfloat16*>(a.packs);
  const int kc = ld / 8;
  for (int q = tid; q < n_k * kc; q += blockDim.x) {
    const int i = q / kc, c = q % kc;
    const uint4 v = *reinterpret_cast<const uint4*>(pk + (long long)i * ld + 8 * c);
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int j = 8 * c + t;
      if (j < n_v) *reinterpret_cast<unsigned short*>(At + tc_off(j, i, sbo)) = bf16_bits(v, t);
    }
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init(&sbar[0], 1);
    mbar_init(&sbar[1], 1);
    fence_barrier_init();
  }
  if (warp == 0) {  // tn <= 64 accumulator columns
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)), "r"(64));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_proxy_async();
  tc_sync();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(tn >> 3) << 17) | (8u << 24);
  const VT* sp = reinterpret_cast<const VT*>(a.spub);
  const VT* wb = reinterpret_cast<const VT*>(a.wbuf);
  VT* rp = reinterpret_cast<VT*>(a.rpub);
  uint32_t phase = 0;
  bool failed = false;
  const int batches = (a.n + tn - 1) / tn;
  auto full = [&](int bt) { return bt < batches && (long long)(bt + 1) * tn <= a.n; };
  uint32_t sphase = 0;   // bit sb: the phase of buffer sb's barrier to wait for
  uint32_t pending = 0;  // bit sb: a copy into buffer sb issued and not yet awaited
  auto stage_copy = [&](int bt, int sb) {
    if (tid == 0) {
      fence_proxy_async();  // the buffer's last reads (generic) before the copies' writes (async)
      unsigned char* dst = stage0 + (size_t)sb * sbytes;
      mbar_expect_tx(&sbar[sb], sbytes);
      bulk_g2s(dst, sp + (long long)bt * tn * n_x, sx, &sbar[sb]);
      bulk_g2s(dst + sx, wb + (long long)bt * tn * n_k, sbytes - sx, &sbar[sb]);
    }
    pending |= 1u << sb;
  };
  if (full(blockIdx.x)) stage_copy(blockIdx.x, 0);
  int it = 0;
  for (int bt = blockIdx.x; bt < batches && !failed; bt += gridDim.x, ++it) {
    const long long m0 = (long long)bt * tn;
    const int nb = min(tn, a.n - (int)m0);
    const int sb = it & 1;
    const bool staged = full(bt);
    // the next batch's rows into the other buffer, whose last reads ended at the previous batch's barriers
    if (full(bt + (int)gridDim.x)) stage_copy(bt + (int)gridDim.x, sb ^ 1);
    if (staged) {
      if (mbar_wait(&sbar[sb], (sphase >> sb) & 1u)) {
        sphase ^= 1u << sb;
        pending &= ~(1u << sb);
      } else {
        failed = true;
      }
      if (__syncthreads_or(failed)) {
        failed = true;
        break;
      }
    }
    // Y: row b = [s; psi] of node m0 + b, bfloat16 (columns n_k .. Kq - 1 stay zero)
    const float* ss = reinterpret_cast<const float*>(stage0 + (size_t)sb * sbytes);
    const float* sw = reinterpret_cast<const float*>(stage0 + (size_t)sb * sbytes + sx);
    for (int q = tid; q < tn * n_k; q += blockDim.x) {
      const int b = q / n_k, i = q % n_k;
      float v;
      if (staged)
        v = i < n_x ? ss[b * n_x + i] : sw[q];
      else
        v = b < nb ? (float)(i < n_x ? sp[(m0 + b) * n_x + i] : wb[(m0 + b) * n_k + i]) : 0.f;
      *reinterpret_cast<__nv_bfloat16*>(Bm + tc_off(b, i, sbo)) = __float2bfloat16_rn(v);
    }
    fence_proxy_async();
    tc_sync();
    if (tid == 0) {
      for (int ks = 0; ks < Kq / 16; ++ks)
        umma_bf16(tmem, umma_desc(smem_u32(At) + ks * 2 * kTcCore, kTcCore, sbo),
                  umma_desc(smem_u32(Bm) + ks * 2 * kTcCore, kTcCore, sbo), idesc, ks > 0);
      umma_commit(bar);
    }
    if (!mbar_wait(bar, phase)) failed = true;
    phase ^= 1;
    if (__syncthreads_or(failed)) {
      failed = true;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // g: warp w reads rows 32 (w mod 4) .. + 31 of D (the entries of g), one column per node
    const int j = 32 * qw + lane;
    for (int c0 = 16 * hc; c0 < tn; c0 += 32) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(32 * qw) << 16) + c0, v);
      if (j < n_v) {
#pragma unroll
        for (int t = 0; t < 16; ++t)
          if (c0 + t < nb) rp[(m0 + c0 + t) * n_v + j] = (VT)v[t];
      }
    }
    tc_sync();  // Y and the accumulators are free for the next batch
  }
  if (failed && tid == 0) {
    a.flags[1] = SMPC_ETIMEOUT;
    mbar_wait(bar, phase ^ 1);  // bounded: let the MMAs in flight finish before freeing tensor memory
  }
  if (failed)  // bounded: let the staging copies in flight land before the CTA's shared memory goes
    for (int sb = 0; sb < 2; ++sb)
      if ((pending >> sb) & 1u) mbar_wait(&sbar[sb], (sphase >> sb) & 1u);
  tc_sync();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(64));
}

int optin_smem() {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return optin > 0 ? optin : 232448;
}

template <typename VT, typename MT>
LaunchCfg config_t(const IterArgs& a, int num_sms, int S_max, int schedule, int tc_width = 0) {
  LaunchCfg c;
  const int optin = optin_smem();
  c.schedule = schedule;
  c.block = kThreads;
  const bool fits_threads = a.n_k <= kThreads && a.n_v <= kThreads;  // one thread per entry
  if (schedule == SCHED_CHAIN) {
    int S = S_max;
    while (S > 1 && iter_smem_bytes<MT>(S, a.n_x, a.n_u, a.n_v) > (size_t)optin) --S;
    c.stages = S;
    c.smem = iter_smem_bytes<MT>(S, a.n_x, a.n_u, a.n_v);
    if (c.smem > (size_t)optin || !fits_threads || a.A) c.stages = 0;  // its chain pass has no A' step
    c.grid = a.n_chains < num_sms ? a.n_chains : num_sms;
    if (c.grid < 1) c.grid = 1;
    return c;
  }
  c.stages = fits_threads ? 1 : 0;
  if (schedule == SCHED_HYBRID) {
    const LaunchCfg ch = config_t<VT, MT>(a, num_sms, S_max, SCHED_CHAIN);
    c.grid_chain = ch.grid;
    c.stages_chain = ch.stages;
    c.smem_chain = ch.smem;
    if (ch.stages < 1) c.stages = 0;
  }
  if (schedule == SCHED_FUSED) {  // chain_bwd: kBT threads, as many pack slots as fit
    int S = S_max;
    while (S > 1 && bwd_smem_bytes<MT>(S, a.n_x, a.n_u, a.n_v) + 256 > (size_t)optin) --S;
    c.stages_chain = S;
    c.smem_chain = bwd_smem_bytes<MT>(S, a.n_x, a.n_u, a.n_v);
    c.grid_chain = a.n_chains < num_sms ? a.n_chains : num_sms;
    if (c.grid_chain < 1) c.grid_chain = 1;
    if (c.smem_chain + 256 > (size_t)optin || 2 * a.n_k > kBT || a.n_v > kBT || a.A) c.stages = 0;
  }
  c.smem_prox = iter_smem_bytes<MT>(0, a.n_x, a.n_u, a.n_v);  // barriers + vectors, no pack slot
  c.smem_pstage = c.smem_prox + (size_t)kWarps * prox_stage_bytes<VT>(a.n_x, a.n_u);
  if (c.smem_pstage + 5 * kThreads * sizeof(double) + 1024 > (size_t)optin) c.stages = 0;
  c.grid_prox = (a.n + kWarps - 1) / kWarps;  // one warp per node
  if (c.grid_prox > 8 * num_sms) c.grid_prox = 8 * num_sms;
  c.grid_scan = a.n_chains < 4 * num_sms ? a.n_chains : 4 * num_sms;
  c.grid_fwd = a.n_top + a.n_chains < 8 * num_sms ? a.n_top + a.n_chains : 8 * num_sms;
  c.grid_mv = a.n < num_sms ? a.n : num_sms;
  if (c.grid_scan < 1) c.grid_scan = 1;
  // launches with h_a (anchored solves) come from bfloat16 factors' configurations, or from
  // configurations made with a.ha set
  c.smem_fwd = fwd_smem_bytes<VT>(a.n_k, std::is_same<MT, __nv_bfloat16>::value || a.ha != nullptr);
  if (c.smem_fwd + 1024 > (size_t)optin) c.stages = 0;
  int S = kMaxSlots;
  while (S > 0 && iter_smem_bytes<MT>(S, a.n_x, a.n_u, a.n_v, false) > (size_t)optin) --S;
  c.s_gt = S;
  c.smem_gt = iter_smem_bytes<MT>(S > 0 ? S : 1, a.n_x, a.n_u, a.n_v, false);
  S = kMaxSlots;
  while (S > 0 && iter_smem_bytes<MT>(S, a.n_x, a.n_u, a.n_v, true) > (size_t)optin) --S;
  c.s_dh = S;
  c.smem_dh = iter_smem_bytes<MT>(S > 0 ? S : 1, a.n_x, a.n_u, a.n_v, true);
  if (c.s_gt < 1 || c.s_dh < 1) c.stages = 0;
  // shared pack: kNB nodes per pass when the pack and the staging fit
  c.multi_gt = c.multi_dh = false;
  c.tc = false;
  if (a.pack_stride == 0 && std::is_same<MT, __nv_bfloat16>::value && tc_fits(a.n_x, a.n_u, a.n_v) &&
      tc_smem_bytes(a.n_v, kTcMaxN) + 256 <= (size_t)optin) {
    // the widest GEMM (16, 32 or 64 nodes) that still gives every SM a batch
    c.tc = true;
    if (tc_width == 16 || tc_width == 32 || tc_width == 64) {
      c.tn = tc_width;  // chosen by timing when the factor was built
    } else {
      c.tn = 16;  // the widest GEMM that still gives every SM two batches
      while (c.tn < kTcMaxN && a.n >= 2 * c.tn * num_sms) c.tn *= 2;
    }
    c.smem_tc = tc_smem_bytes(a.n_v, c.tn);
    const int batches = (a.n + c.tn - 1) / c.tn;
    c.grid_tc = batches < num_sms ? batches : num_sms;
    c.smem_gt_tc = gt_smem_bytes(a.n_x, a.n_k, c.tn);  // [Bbar; L]' y on the tensor cores when it fits
    c.tc_gt = c.smem_gt_tc + 256 <= (size_t)optin;
  }
  if (a.pack_stride == 0) {
    c.smem_mgt = multi_smem_bytes<MT>(a.n_x, a.n_u, a.n_v, false);
    c.smem_mdh = multi_smem_bytes<MT>(a.n_x, a.n_u, a.n_v, true);
    c.multi_gt = c.smem_mgt + 256 <= (size_t)optin;  // room for the kernel's static shared memory
    c.multi_dh = c.smem_mdh + 256 <= (size_t)optin;
    const int batches = (a.n + kNB - 1) / kNB;
    c.grid_multi = batches < num_sms ? batches : num_sms;
  }
  return c;
}

// Launch with programmatic dependent launch allowed (dep): the kernel may be scheduled
// while the stream's previous kernel drains; it calls grid_dep_sync before any access.
template <typename... KArgs, typename... Args>
void launch_dep(void (*kern)(KArgs...), int grid, int block, size_t smem, cudaStream_t s, bool dep, Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = dep ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kern, args...);
}

template <typename VT, typename MT>
int launch_t(const IterArgs& a, const LaunchCfg& c, int nu, int mode, cudaStream_t s) {
  // once per process and instantiation; thread-safe (solves may run on several threads).
  // Each kernel may use the opt-in shared memory minus its static shared memory.
  static const bool attr_set = [] {
    const int optin = optin_smem();
    auto allow = [optin](auto fn) {
      cudaFuncAttributes at{};
      if (cudaFuncGetAttributes(&at, fn) == cudaSuccess)
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)at.sharedSizeBytes);
    };
    allow(apg_iter<VT, MT>);
    allow(chain_bwd<VT, MT>);
    allow(node_mv<VT, MT, false>);
    allow(node_mv<VT, MT, true>);
    allow(prox_node<VT, MT>);
    allow(fwd_scan<VT, MT>);
    allow(node_mv_shared<VT, MT, false>);
    allow(node_mv_shared<VT, MT, true>);
    if constexpr (std::is_same<MT, __nv_bfloat16>::value) {
      allow(node_mv_tc<VT>);
      allow(node_gt_tc<VT>);
    }
    cudaGetLastError();  // a refused attribute surfaces at the launch, not here
    return true;
  }();
  (void)attr_set;
  int ev = 0;
  const bool dep = c.events == nullptr;  // stage events between the kernels would cut the overlap anyway
  auto mark = [&]() {
    if (c.events) cudaEventRecord(c.events[ev++], s);
  };
  mark();
  if (c.schedule == SCHED_CHAIN) {
    launch_dep(apg_iter<VT, MT>, c.grid, c.block, c.smem, s, dep, a, c.stages, nu, mode);
    mark();
    return check_launch("apg_iter");
  }
  if ((mode & MODE_PROX) && nu >= 1) {
    launch_dep(fwd_scan<VT, MT>, c.grid_fwd, c.block, c.smem_fwd, s, dep, a, nu, mode);
    mark();
  }
  launch_dep(prox_node<VT, MT>, c.grid_prox, c.block, c.smem_pstage, s, dep, a, nu, mode);
  mark();
  if ((mode & MODE_BWD) && c.schedule == SCHED_FUSED) {
    // the whole backward sweep (s, [Bbar; L]'[s; psi], r, Lambda r / (2 p) and [Bbar; L] delta)
    // along the chains and up the top nodes: every pack is read once per iteration
    launch_dep(chain_bwd<VT, MT>, c.grid_chain, kBT, c.smem_chain, s, dep, a, c.stages_chain, nu,
               (mode & ~MODE_PROX) | MODE_WREADY);
    mark();
  } else if ((mode & MODE_BWD) && c.schedule == SCHED_HYBRID) {
    // s, [Bbar; L]'[s; psi] and r along the chains and up the top nodes, r of every node out
    launch_dep(apg_iter<VT, MT>, c.grid_chain, c.block, c.smem_chain, s, dep, a, c.stages_chain, nu,
                                                                 (mode & ~MODE_PROX) | MODE_GT | MODE_WREADY);
    mark();
    if constexpr (std::is_same<MT, __nv_bfloat16>::value) {
      if (c.tc && (mode & MODE_DELTA)) {
        launch_dep(node_mv_tc<VT>, c.grid_tc, kTcThreads, c.smem_tc, s, dep, a, c.tn, nu, mode);
      } else if (c.multi_dh) {
        launch_dep(node_mv_shared<VT, MT, true>, c.grid_multi, c.block, c.smem_mdh, s, dep, a, nu, mode);
      } else {
        launch_dep(node_mv<VT, MT, true>, c.grid_mv, c.block, c.smem_dh, s, dep, a, c.s_dh, nu, mode);
      }
    } else {
      if (c.multi_dh)
        launch_dep(node_mv_shared<VT, MT, true>, c.grid_multi, c.block, c.smem_mdh, s, dep, a, nu, mode);
      else
        launch_dep(node_mv<VT, MT, true>, c.grid_mv, c.block, c.smem_dh, s, dep, a, c.s_dh, nu, mode);
    }
    mark();
  } else if (mode & MODE_BWD) {
    launch_dep(scan_kernel<VT>, c.grid_scan, c.block, 0, s, dep, a, 0, nu, mode);
    mark();
    bool gt_done = false;
    if constexpr (std::is_same<MT, __nv_bfloat16>::value) {
      if (c.tc && c.tc_gt && (mode & MODE_DELTA)) {
        launch_dep(node_gt_tc<VT>, c.grid_tc, kTcThreads, c.smem_gt_tc, s, dep, a, c.tn, nu, mode);
        gt_done = true;
      }
    }
    if (gt_done)
      ;
    else if (c.multi_gt)
      launch_dep(node_mv_shared<VT, MT, false>, c.grid_multi, c.block, c.smem_mgt, s, dep, a, nu, mode);
    else
      launch_dep(node_mv<VT, MT, false>, c.grid_mv, c.block, c.smem_gt, s, dep, a, c.s_gt, nu, mode);
    mark();
    launch_dep(scan_kernel<VT>, c.grid_scan, c.block, 0, s, dep, a, 1, nu, mode);
    mark();
    if constexpr (std::is_same<MT, __nv_bfloat16>::value) {
      if (c.tc && (mode & MODE_DELTA)) {
        launch_dep(node_mv_tc<VT>, c.grid_tc, kTcThreads, c.smem_tc, s, dep, a, c.tn, nu, mode);
      } else if (c.multi_dh) {
        launch_dep(node_mv_shared<VT, MT, true>, c.grid_multi, c.block, c.smem_mdh, s, dep, a, nu, mode);
      } else {
        launch_dep(node_mv<VT, MT, true>, c.grid_mv, c.block, c.smem_dh, s, dep, a, c.s_dh, nu, mode);
      }
    } else {
      if (c.multi_dh)
        launch_dep(node_mv_shared<VT, MT, true>, c.grid_multi, c.block, c.smem_mdh, s, dep, a, nu, mode);
      else
        launch_dep(node_mv<VT, MT, true>, c.grid_mv, c.block, c.smem_dh, s, dep, a, c.s_dh, nu, mode);
    }
    mark();
  }
  return check_launch("node-parallel iteration");
}

}  // namespace

size_t vec_size(int prec) { return prec == SMPC_FP64 ? sizeof(double) : sizeof(float); }
size_t mat_size(int prec) {
  return prec == SMPC_FP64 ? sizeof(double) : prec == SMPC_FP32 ? sizeof(float) : sizeof(__nv_bfloat16);
}
long long pack_entries(int prec, int n_k, int n_v) {
  switch (prec) {
    case SMPC_FP64: return kpad<double>(n_k, n_v) + lpad<double>(n_v);
    case SMPC_FP32: return kpad<float>(n_k, n_v) + lpad<float>(n_v);
    default: return kpad<__nv_bfloat16>(n_k, n_v) + lpad<__nv_bfloat16>(n_v);
  }
}

LaunchCfg iter_config(int prec, const IterArgs& a, int num_sms, int schedule, int tc_width) {
  switch (prec) {
    case SMPC_FP64: return config_t<double, double>(a, num_sms, 1, schedule);
    case SMPC_FP32: return config_t<float, float>(a, num_sms, 2, schedule);
    default: return config_t<float, __nv_bfloat16>(a, num_sms, 4, schedule, tc_width);
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

int launch_cut_sums(int prec, const IterArgs& a, int n_cut, const int* cut_off, const int* cut_heads, void* out,
                    void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n_cut <= 0) return SMPC_OK;
  const int grid = n_cut < 1024 ? n_cut : 1024;
  if (prec == SMPC_FP64)
    cut_sums_kernel<double><<<grid, 256, 0, s>>>(a, n_cut, cut_off, cut_heads, (double*)out);
  else
    cut_sums_kernel<float><<<grid, 256, 0, s>>>(a, n_cut, cut_off, cut_heads, (float*)out);
  return check_launch("cut_sums");
}

int launch_cut_scatter(int prec, const IterArgs& a, int n_cut, const int* chl_off, const int* chl, const void* in,
                       void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n_cut <= 0) return SMPC_OK;
  const int grid = n_cut < 1024 ? n_cut : 1024;
  if (prec == SMPC_FP64)
    cut_scatter_kernel<double><<<grid, 256, 0, s>>>(a, n_cut, chl_off, chl, (const double*)in);
  else
    cut_scatter_kernel<float><<<grid, 256, 0, s>>>(a, n_cut, chl_off, chl, (const float*)in);
  return check_launch("cut_scatter");
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
