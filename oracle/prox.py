"""Proximal operators of g (Sec. IV-C and App. C).

g(t) = sum_n  mu_S,n dist(vsigma_n | C_s) + gamma_d dist(zeta_n | C_1) + delta(psi_n | U)
with C_s = {x >= x_s}, C_1 = {x_min <= x <= x_max}, U = {u_min <= u <= u_max} and
the Euclidean distance over the node's whole n_x-vector (eq. cost:non-smooth).

App. C gives, for g = mu dist(. | C) and step gamma,
    prox_{gamma g}(v) = v + gamma mu (P_C(v) - v) / dist(v | C)   if dist(v | C) > gamma mu,
                        P_C(v)                                     otherwise.
(The printed formula drops the factor gamma mu in the first branch; with it the
two branches meet at dist = gamma mu, as the prox of a distance must.)  The prox of
an indicator is the projection (App. C).  By the separable-sum property (eq.
separable-sum-property) each node block is handled on its own.
"""
from __future__ import annotations

import numpy as np


def prox_dist(v, P, gamma_mu):
    """Row-wise prox of gamma_mu * dist(. | C) given P = P_C(v); gamma_mu per row."""
    v = np.asarray(v, float)
    P = np.asarray(P, float)
    gm = np.broadcast_to(np.asarray(gamma_mu, float), (v.shape[0],))
    dist = np.sqrt(np.sum((v - P) ** 2, axis=1))
    out = P.copy()
    far = dist > gm
    out[far] = v[far] + (gm[far] / dist[far])[:, None] * (P[far] - v[far])
    return out


def prox_box(v, lo, hi):
    return np.minimum(np.maximum(np.asarray(v, float), lo), hi)


def prox_g(v_s, v_z, v_p, cost, mu_s, step_s, step_z):
    """Blockwise prox of g / step at (v_s, v_z, v_p): thresholds mu / step per node."""
    t_s = prox_dist(v_s, np.maximum(v_s, cost["x_s"]), mu_s / step_s)
    t_z = prox_dist(v_z, prox_box(v_z, cost["x_min"], cost["x_max"]), cost["gamma_d"] / step_z)
    t_p = prox_box(v_p, cost["u_min"], cost["u_max"])
    return t_s, t_z, t_p
