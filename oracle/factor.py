"""Elimination of the input-disturbance coupling and the factor step.

App. A: the affine set {u : E u + E_d d = 0} is parametrised as u = L v + u_hat(d)
with the columns of L spanning null(E) (eq. new:decision); B_bar = B L,
R_hat = W_u L, R_bar = L' R_hat.
App. B (eq. optimal matrices control): Lambda = -R_bar^{-1} (through a Cholesky
factorisation of R_bar), Phi = Lambda B_bar', Psi = Lambda L'.  The paper prints
"Psi = Lambda L"; only L' (n_u x n_v -> n_v x n_u) matches the dimensions of
Psi psi_tilde in Algorithm 1.

u_hat(d) is taken as the minimum-norm solution -E^+ E_d d; any particular
solution gives the same u, x, y (L and u_hat are not unique, App. A).
"""
from __future__ import annotations

from types import SimpleNamespace

import numpy as np


def factor(net, cost, rank_tol=1e-10):
    A = np.asarray(net["A"], float)
    B = np.asarray(net["B"], float)
    Gd = np.asarray(net["Gd"], float)
    E = np.asarray(net["E"], float)
    Ed = np.asarray(net["Ed"], float)
    W_u = np.asarray(cost["W_u"], float)
    n_u = B.shape[1]
    if E.shape[0] > 0:
        _, S, Vt = np.linalg.svd(E)
        rank = int(np.sum(S > rank_tol * max(1.0, S[0])))
        L = Vt[rank:].T                      # orthonormal basis of null(E)
        P_u = -np.linalg.pinv(E) @ Ed        # u_hat(d) = P_u d
    else:
        L = np.eye(n_u)
        P_u = np.zeros((n_u, Ed.shape[1]))
    B_bar = B @ L
    R_hat = W_u @ L
    R_bar = L.T @ R_hat
    C = np.linalg.cholesky(R_bar)            # R_bar = C C'
    # R_bar^{-1} from the Cholesky factor: solve C Z = I, then C' X = Z
    Z = np.linalg.solve(C, np.eye(R_bar.shape[0]))
    R_bar_inv = np.linalg.solve(C.T, Z)
    Lam = -R_bar_inv
    Phi = Lam @ B_bar.T
    Psi = Lam @ L.T
    return SimpleNamespace(A=A, B=B, Gd=Gd, E=E, Ed=Ed, W_u=W_u, L=L, P_u=P_u,
                           B_bar=B_bar, R_hat=R_hat, R_bar=R_bar, Lam=Lam, Phi=Phi, Psi=Psi,
                           n_x=A.shape[0], n_u=n_u, n_v=L.shape[1], n_d=Gd.shape[1])
