"""Per-step vectors of the solve step (App. A).

For node n at stage j with parent pi(n) and children C(n):

  d_n       = d_hat_j + eps_n                              (eq. demand:tree)
  u_hat_n   = u_hat(d_n)                                   (eq. new:decision)
  e_n       = B u_hat_n + G_d d_n                          (eq. appendix:dist)
  alpha_bar_j = L' W_alpha (alpha_1 + alpha_{2,j})         (App. A; the printed
              "(...) L" is the transpose forced by the dimensions)
  p_bar_n   = p_n + sum_{c in C(n)} p_c
  beta_n    = p_n alpha_bar_j + 2 R_hat' (p_bar_n u_hat_n - p_n u_hat_pi(n)
                                          - sum_{c in C(n)} p_c u_hat_c)

with u_hat_pi(root) := q, the previous input u_{-1}.  This beta is the linear
coefficient obtained by expanding eq. cost:delta into eq. new:stage:cost.  The
printed eq. appendix:beta carries an extra factor p_n on the R_hat term and no
p_n on u_hat_pi; the expansion does not produce them, and the dense KKT test in
the test suite fails with the printed form.
"""
from __future__ import annotations

from types import SimpleNamespace

import numpy as np


def cost_update(fac, cost, tree, alpha2, dhat, eps, q):
    n = tree.n
    stage = tree.stage
    parent = tree.parent
    p = tree.prob
    d = np.asarray(dhat, float)[stage] + np.asarray(eps, float)
    u_hat = d @ fac.P_u.T
    e = u_hat @ fac.B.T + d @ fac.Gd.T
    alpha_bar = (cost["W_alpha"] * (np.asarray(cost["alpha1"], float)[None, :]
                                    + np.asarray(alpha2, float))) @ fac.L
    p_bar = p.copy()
    child_u = np.zeros_like(u_hat)
    for m in range(1, n):                    # children summed in index order
        p_bar[parent[m]] += p[m]
        child_u[parent[m]] += p[m] * u_hat[m]
    u_hat_par = np.empty_like(u_hat)
    u_hat_par[0] = np.asarray(q, float)
    u_hat_par[1:] = u_hat[parent[1:]]
    beta = (p[:, None] * alpha_bar[stage]
            + 2.0 * (p_bar[:, None] * u_hat - p[:, None] * u_hat_par - child_u) @ fac.R_hat)
    return SimpleNamespace(d=d, u_hat=u_hat, e=e, alpha_bar=alpha_bar, p_bar=p_bar, beta=beta)
