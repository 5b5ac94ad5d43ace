"""Dual Hessian, Lipschitz constant and diagonal (Jacobi) scaling on small trees.

The dual gradient is -H z(w) (Sec. IV-A); z(w) is affine in w, so the dual
Hessian is H_D = -d(H z)/dw, a symmetric positive semidefinite matrix.  Here it
is formed column by column from Algorithm 1 run with the affine data removed
(beta = u_hat = e = 0, x_0 = 0), which leaves exactly the linear part.

Sec. IV-D: lambda = 1 / L_{H_D} with L_{H_D} the largest eigenvalue of the
(scaled) dual Hessian; the diagonal preconditioner approximates H_D by a
diagonal matrix and scales the dual by its inverse square root.  Reading used
here: Jacobi scaling d_i = 1 / (H_D)_ii on the input block (elementwise), and one
scalar per distance block, 1 / mean of the block's diagonal, so that the scaled
prox of a distance keeps its closed form.  An input entry that the coupling fixes
(a zero row of L: zero curvature) takes the mean diagonal of its node's other
input entries.  The paper computes these on one
branch; this oracle computes them on the whole (small) tree.
"""
from __future__ import annotations

from types import SimpleNamespace

import numpy as np

from .solve_step import solve_step


def dense_dual_hessian(fac, tree):
    n, n_x, n_u, n_v = tree.n, fac.n_x, fac.n_u, fac.n_v
    blk = 2 * n_x + n_u
    zero = SimpleNamespace(beta=np.zeros((n, n_v)), u_hat=np.zeros((n, n_u)), e=np.zeros((n, n_x)))
    M = np.zeros((n * blk, n * blk))
    for k in range(n * blk):
        w = np.zeros((n, blk))
        w.flat[k] = 1.0
        x, u = solve_step(fac, tree, zero, w[:, :n_x], w[:, n_x:2 * n_x], w[:, 2 * n_x:], np.zeros(n_x))
        M[:, k] = -np.concatenate([x, x, u], axis=1).ravel()
    return M


def lipschitz_dense(M):
    return float(np.linalg.eigvalsh(0.5 * (M + M.T))[-1])


def jacobi_steps(fac, tree, M=None):
    """Per-entry steps lambda * d of the Jacobi-scaled iteration (Sec. IV-D reading)."""
    n, n_x, n_u = tree.n, fac.n_x, fac.n_u
    blk = 2 * n_x + n_u
    if M is None:
        M = dense_dual_hessian(fac, tree)
    diag = np.diag(M).reshape(n, blk)
    d_s = 1.0 / diag[:, :n_x].mean(axis=1)
    d_z = 1.0 / diag[:, n_x:2 * n_x].mean(axis=1)
    dp_diag = diag[:, 2 * n_x:]
    # an input entry fixed by the coupling (zero row of L) has zero curvature; it
    # takes the mean curvature of the other input entries of its node
    live = dp_diag > 1e-12 * dp_diag.max(axis=1, keepdims=True)
    fill = np.where(live, dp_diag, 0.0).sum(axis=1, keepdims=True) / live.sum(axis=1, keepdims=True)
    d_p = 1.0 / np.where(live, dp_diag, fill)
    dvec = np.concatenate([np.repeat(d_s[:, None], n_x, 1), np.repeat(d_z[:, None], n_x, 1), d_p], axis=1).ravel()
    sq = np.sqrt(dvec)
    lam = 1.0 / lipschitz_dense(sq[:, None] * M * sq[None, :])
    return {"s": lam * d_s, "z": lam * d_z, "p": lam * d_p, "lambda": lam,
            "d_s": d_s, "d_z": d_z, "d_p": d_p}
