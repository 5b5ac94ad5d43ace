// Host float64 factor step (App. A and App. B): null-space elimination of the
// input-disturbance coupling and the inverse of R_bar through its Cholesky
// factor.  Plain loops; the sizes are those of the network (n_u ~ 100).
#include <cmath>
#include <vector>

#include "smpc_internal.h"

namespace smpc {
namespace {

// C (m x n) = A (m x k) * B (k x n), row-major
void gemm(const double* A, const double* B, double* C, int m, int k, int n, bool transA = false) {
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0;
      for (int p = 0; p < k; ++p) s += (transA ? A[p * m + i] : A[i * k + p]) * B[p * n + j];
      C[i * n + j] = s;
    }
}

// In-place Cholesky A = G G' (lower, row-major n x n).  Returns false if not SPD.
bool cholesky(std::vector<double>& A, int n) {
  for (int j = 0; j < n; ++j) {
    double d = A[j * n + j];
    for (int k = 0; k < j; ++k) d -= A[j * n + k] * A[j * n + k];
    if (!(d > 0)) return false;
    d = std::sqrt(d);
    A[j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double s = A[i * n + j];
      for (int k = 0; k < j; ++k) s -= A[i * n + k] * A[j * n + k];
      A[i * n + j] = s / d;
    }
    for (int k = j + 1; k < n; ++k) A[j * n + k] = 0;
  }
  return true;
}

// Solve (G G') X = B for X (n x m) given the Cholesky factor G.
void chol_solve(const std::vector<double>& G, int n, std::vector<double>& B, int m) {
  for (int c = 0; c < m; ++c) {
    for (int i = 0; i < n; ++i) {  // forward G z = b
      double s = B[i * m + c];
      for (int k = 0; k < i; ++k) s -= G[i * n + k] * B[k * m + c];
      B[i * m + c] = s / G[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {  // backward G' x = z
      double s = B[i * m + c];
      for (int k = i + 1; k < n; ++k) s -= G[k * n + i] * B[k * m + c];
      B[i * m + c] = s / G[i * n + i];
    }
  }
}

// Householder QR of M (rows x cols, rows >= cols); returns the full orthogonal Q
// (rows x rows) and the diagonal of R.
void householder_q(std::vector<double> M, int rows, int cols, std::vector<double>& Q, std::vector<double>& rdiag) {
  Q.assign((size_t)rows * rows, 0.0);
  for (int i = 0; i < rows; ++i) Q[i * rows + i] = 1.0;
  rdiag.assign(cols, 0.0);
  std::vector<double> v(rows);
  for (int k = 0; k < cols; ++k) {
    double nrm = 0;
    for (int i = k; i < rows; ++i) nrm += M[i * cols + k] * M[i * cols + k];
    nrm = std::sqrt(nrm);
    if (nrm == 0) {
      rdiag[k] = 0;
      continue;
    }
    const double alpha = M[k * cols + k] > 0 ? -nrm : nrm;
    for (int i = 0; i < rows; ++i) v[i] = (i < k) ? 0 : M[i * cols + k];
    v[k] -= alpha;
    double vv = 0;
    for (int i = k; i < rows; ++i) vv += v[i] * v[i];
    if (vv == 0) {
      rdiag[k] = alpha;
      continue;
    }
    // M <- (I - 2 v v'/vv) M
    for (int j = k; j < cols; ++j) {
      double s = 0;
      for (int i = k; i < rows; ++i) s += v[i] * M[i * cols + j];
      s *= 2.0 / vv;
      for (int i = k; i < rows; ++i) M[i * cols + j] -= s * v[i];
    }
    // Q <- Q (I - 2 v v'/vv)
    for (int r = 0; r < rows; ++r) {
      double s = 0;
      for (int i = k; i < rows; ++i) s += Q[r * rows + i] * v[i];
      s *= 2.0 / vv;
      for (int i = k; i < rows; ++i) Q[r * rows + i] -= s * v[i];
    }
    rdiag[k] = M[k * cols + k];
  }
}

}  // namespace

int host_factor(const smpc_network& net, const double* W_u, HostFactor& f) {
  const int n_x = net.n_x, n_u = net.n_u, n_d = net.n_d, n_e = net.n_e;
  f.n_x = n_x;
  f.n_u = n_u;
  f.n_d = n_d;
  f.n_e = n_e;
  // L: columns n_e .. n_u-1 of Q from E' = Q R (they span null(E) when E has full row rank)
  if (n_e > 0) {
    std::vector<double> Et((size_t)n_u * n_e);
    double emax = 0;
    for (int i = 0; i < n_e; ++i)
      for (int j = 0; j < n_u; ++j) {
        Et[j * n_e + i] = net.E[i * n_u + j];
        emax = std::fmax(emax, std::fabs(net.E[i * n_u + j]));
      }
    if (n_e >= n_u) {
      set_error("E has n_e = %d >= n_u = %d rows: no free inputs", n_e, n_u);
      return SMPC_EINVAL;
    }
    std::vector<double> Q, rd;
    householder_q(Et, n_u, n_e, Q, rd);
    for (int k = 0; k < n_e; ++k)
      if (!(std::fabs(rd[k]) > 1e-10 * std::fmax(1.0, emax))) {
        set_error("E is rank deficient (pivot %d = %g)", k, rd[k]);
        return SMPC_EINVAL;
      }
    f.n_v = n_u - n_e;
    f.L.assign((size_t)n_u * f.n_v, 0.0);
    for (int i = 0; i < n_u; ++i)
      for (int j = 0; j < f.n_v; ++j) f.L[i * f.n_v + j] = Q[i * n_u + n_e + j];
    // Pu = -E' (E E')^{-1} Ed  (minimum-norm particular solution of E u + Ed d = 0)
    std::vector<double> EEt((size_t)n_e * n_e);
    for (int i = 0; i < n_e; ++i)
      for (int j = 0; j < n_e; ++j) {
        double s = 0;
        for (int k = 0; k < n_u; ++k) s += net.E[i * n_u + k] * net.E[j * n_u + k];
        EEt[i * n_e + j] = s;
      }
    if (!cholesky(EEt, n_e)) {
      set_error("E E' is not positive definite");
      return SMPC_EINVAL;
    }
    std::vector<double> Z(net.Ed, net.Ed + (size_t)n_e * n_d);
    chol_solve(EEt, n_e, Z, n_d);
    f.Pu.assign((size_t)n_u * n_d, 0.0);
    for (int i = 0; i < n_u; ++i)
      for (int j = 0; j < n_d; ++j) {
        double s = 0;
        for (int k = 0; k < n_e; ++k) s += net.E[k * n_u + i] * Z[k * n_d + j];
        f.Pu[i * n_d + j] = -s;
      }
  } else {
    f.n_v = n_u;
    f.L.assign((size_t)n_u * n_u, 0.0);
    for (int i = 0; i < n_u; ++i) f.L[i * n_u + i] = 1.0;
    f.Pu.assign((size_t)n_u * n_d, 0.0);
  }
  const int n_v = f.n_v;
  f.Bbar.resize((size_t)n_x * n_v);
  gemm(net.B, f.L.data(), f.Bbar.data(), n_x, n_u, n_v);
  f.Rhat.resize((size_t)n_u * n_v);
  gemm(W_u, f.L.data(), f.Rhat.data(), n_u, n_u, n_v);
  f.Rbar.resize((size_t)n_v * n_v);
  gemm(f.L.data(), f.Rhat.data(), f.Rbar.data(), n_v, n_u, n_v, /*transA=*/true);
  for (int i = 0; i < n_v; ++i)  // exact symmetry
    for (int j = 0; j < i; ++j) {
      const double s = 0.5 * (f.Rbar[i * n_v + j] + f.Rbar[j * n_v + i]);
      f.Rbar[i * n_v + j] = f.Rbar[j * n_v + i] = s;
    }
  std::vector<double> G = f.Rbar;
  if (!cholesky(G, n_v)) {
    set_error("R_bar = L' W_u L is not positive definite (W_u not SPD?)");
    return SMPC_EINVAL;
  }
  std::vector<double> Rinv((size_t)n_v * n_v, 0.0);
  for (int i = 0; i < n_v; ++i) Rinv[i * n_v + i] = 1.0;
  chol_solve(G, n_v, Rinv, n_v);
  f.Lam.resize((size_t)n_v * n_v);
  for (int i = 0; i < n_v; ++i)
    for (int j = 0; j < n_v; ++j) f.Lam[i * n_v + j] = -0.5 * (Rinv[i * n_v + j] + Rinv[j * n_v + i]);
  // Pe = B Pu + Gd
  f.Pe.resize((size_t)n_x * n_d);
  gemm(net.B, f.Pu.data(), f.Pe.data(), n_x, n_u, n_d);
  for (size_t i = 0; i < f.Pe.size(); ++i) f.Pe[i] += net.Gd[i];
  // Jacobi ingredients: diag(Bbar Rbar^{-1} Bbar') and diag(L Rbar^{-1} L')
  f.diagB.assign(n_x, 0.0);
  f.diagL.assign(n_u, 0.0);
  for (int i = 0; i < n_x; ++i) {
    double s = 0;
    for (int a = 0; a < n_v; ++a)
      for (int b = 0; b < n_v; ++b) s += f.Bbar[i * n_v + a] * Rinv[a * n_v + b] * f.Bbar[i * n_v + b];
    f.diagB[i] = s;
  }
  for (int i = 0; i < n_u; ++i) {
    double s = 0;
    for (int a = 0; a < n_v; ++a)
      for (int b = 0; b < n_v; ++b) s += f.L[i * n_v + a] * Rinv[a * n_v + b] * f.L[i * n_v + b];
    f.diagL[i] = s;
  }
  return SMPC_OK;
}

}  // namespace smpc
