"""Algorithm 1 (solve step): z = argmin_z <z, H'w> + f(z) by dynamic programming.

Reading of the printed algorithm (the indices in it are garbled):
* node n at stage j holds (u_n, x_n = x_{j+1}); its dual block is
  w_n = (vsigma_n, zeta_n, psi_n) and xi_n = vsigma_n + zeta_n (the part of H'w that
  multiplies x_n; the paper writes xi as the pair);
* backward sweep, stages N-1 down to 0, nodes of a stage together:
      s_n     = xi_n + sum_{c in C(n)} q_c
      sigma_n = beta_n + sum_{c in C(n)} r_c
      delta_n = (Phi s_n + Psi psi_n + Lambda sigma_n) / (2 p_n)
      r_n     = sigma_n + B_bar' s_n + L' psi_n        (printed "L psi"; L' by dimensions)
      q_n     = A' s_n                                  (= A' sum(xi + q) of the paper)
  leaves have no children, so their sums are zero (q_N = r_N = 0);
* forward sweep, stages 0 up to N-1:
      v_n = v_pi(n) + delta_n,   u_n = L v_n + u_hat_n,
      x_n = A x_pi(n) + B_bar v_n + e_n,
  with v_pi(root) = 0 and x_pi(root) = p (the measured state).
The previous input q enters only through beta_root (see cost_update).
"""
from __future__ import annotations

import numpy as np


def solve_step(fac, tree, cu, w_s, w_z, w_p, p0, return_internals=False):
    n, n_x, n_u, n_v = tree.n, fac.n_x, fac.n_u, fac.n_v
    parent = tree.parent
    prob = tree.prob
    xi = np.asarray(w_s, float) + np.asarray(w_z, float)
    w_p = np.asarray(w_p, float)
    q_sum = np.zeros((n, n_x))      # sum over children of q_c
    r_sum = np.zeros((n, n_v))      # sum over children of r_c
    delta = np.zeros((n, n_v))
    q = np.zeros((n, n_x))
    r = np.zeros((n, n_v))
    for j in range(tree.horizon - 1, -1, -1):
        S = tree.nodes_at[j]
        s = xi[S] + q_sum[S]
        sigma = cu.beta[S] + r_sum[S]
        delta[S] = (s @ fac.Phi.T + w_p[S] @ fac.Psi.T + sigma @ fac.Lam.T) / (2.0 * prob[S])[:, None]
        r[S] = sigma + s @ fac.B_bar + w_p[S] @ fac.L
        q[S] = s @ fac.A
        if j > 0:                           # children added in index order
            np.add.at(q_sum, parent[S], q[S])
            np.add.at(r_sum, parent[S], r[S])
    v = np.zeros((n, n_v))
    u = np.zeros((n, n_u))
    x = np.zeros((n, n_x))
    for j in range(tree.horizon):
        S = tree.nodes_at[j]
        if j == 0:
            v_par = np.zeros((len(S), n_v))
            x_par = np.broadcast_to(np.asarray(p0, float), (len(S), n_x))
        else:
            v_par = v[parent[S]]
            x_par = x[parent[S]]
        v[S] = v_par + delta[S]
        u[S] = v[S] @ fac.L.T + cu.u_hat[S]
        x[S] = x_par @ fac.A.T + v[S] @ fac.B_bar.T + cu.e[S]
    if return_internals:
        return x, u, {"v": v, "delta": delta, "r": r, "q": q}
    return x, u
