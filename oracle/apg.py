"""Accelerated dual proximal gradient iteration (eq. apg-iteration, Sec. IV-A).

  w^nu     = y^nu + theta_nu (1/theta_{nu-1} - 1)(y^nu - y^{nu-1})      (extrapolation)
  z^nu     = argmin_z <z, H'w^nu> + f(z)                               (Algorithm 1)
  t^nu     = prox_{g/lambda}(w^nu / lambda + H z^nu)
  y^{nu+1} = w^nu + lambda (H z^nu - t^nu)
  theta_{nu+1} = (sqrt(theta_nu^4 + 4 theta_nu^2) - theta_nu^2) / 2
starting from y^0 = y^{-1} (zero unless warm-started) and theta_0 = theta_{-1} = 1.
H z = (x, x, u) node by node (eq. optim:H:operator).

Diagonal preconditioning (Sec. IV-D): scaling the dual by D^{-1/2} (D diagonal,
constant on each distance block so that its prox keeps the closed form) is the
same iteration in the original dual coordinates with the scalar lambda replaced by
per-entry steps lambda_i = lambda d_i: v = w / lambda_i + H z, the prox threshold
of a block becomes mu / lambda_i, and y^{nu+1} = w + lambda_i (H z - t).  ``steps``
is either the scalar lambda or a dict with per-node steps for the two distance
blocks ('s', 'z'; shape (n,)) and per-entry steps for the input block ('p'; (n, n_u)).

Residual (Sec. IV-E): rho = ||H z^nu - t^nu||_inf and its relative form
rho / (1 + max(||H z^nu||_inf, ||t^nu||_inf)).  The ergodic primal average
zbar^nu = (1 - theta_nu) zbar^{nu-1} + theta_nu z^nu is returned as well.
Safety weights mu_S,n default to p_n W_x: l^S is inside the expectation of the
problem statement (eq. Sc-MPC) while the printed g omits the probability.
"""
from __future__ import annotations

from types import SimpleNamespace

import numpy as np

from .prox import prox_g
from .solve_step import solve_step


def theta_sequence(K):
    """theta_{-1}, theta_0, ..., theta_K."""
    th = [1.0, 1.0]
    for _ in range(K):
        t = th[-1]
        th.append(0.5 * (np.sqrt(t ** 4 + 4.0 * t ** 2) - t ** 2))
    return np.array(th)


def _steps(steps, n, n_u):
    if isinstance(steps, dict):
        s = np.asarray(steps["s"], float).reshape(n)
        z = np.asarray(steps["z"], float).reshape(n)
        p = np.broadcast_to(np.asarray(steps["p"], float), (n, n_u))
        return s, z, p
    lam = float(steps)
    return np.full(n, lam), np.full(n, lam), np.full((n, n_u), lam)


def apg(fac, tree, cu, cost, p0, steps, iters, mu_s=None, y0=None, tol=None):
    """Runs `iters` iterations, or stops after the first iterate whose relative
    residual is <= tol (Sec. IV-E); the returned histories end at that iterate."""
    n, n_x, n_u = tree.n, fac.n_x, fac.n_u
    lam_s, lam_z, lam_p = _steps(steps, n, n_u)
    if mu_s is None:
        mu_s = tree.prob * cost["W_x"]
    mu_s = np.broadcast_to(np.asarray(mu_s, float), (n,))
    if y0 is None:
        y_s, y_z, y_p = np.zeros((n, n_x)), np.zeros((n, n_x)), np.zeros((n, n_u))
    else:
        y_s, y_z, y_p = (np.array(a, float) for a in y0)
    yp_s, yp_z, yp_p = y_s.copy(), y_z.copy(), y_p.copy()        # y^{-1} = y^0
    theta = theta_sequence(iters)                                 # theta[nu + 1] = theta_nu
    rho = np.zeros(iters)
    rho_rel = np.zeros(iters)
    xbar = ubar = None
    x = u = t_s = t_z = t_p = None
    for nu in range(iters):
        c = theta[nu + 1] * (1.0 / theta[nu] - 1.0)
        w_s = y_s + c * (y_s - yp_s)
        w_z = y_z + c * (y_z - yp_z)
        w_p = y_p + c * (y_p - yp_p)
        x, u = solve_step(fac, tree, cu, w_s, w_z, w_p, p0)
        v_s = w_s / lam_s[:, None] + x
        v_z = w_z / lam_z[:, None] + x
        v_p = w_p / lam_p + u
        t_s, t_z, t_p = prox_g(v_s, v_z, v_p, cost, mu_s, lam_s, lam_z)
        yp_s, yp_z, yp_p = y_s, y_z, y_p
        y_s = w_s + lam_s[:, None] * (x - t_s)
        y_z = w_z + lam_z[:, None] * (x - t_z)
        y_p = w_p + lam_p * (u - t_p)
        res = max(np.abs(x - t_s).max(), np.abs(x - t_z).max(), np.abs(u - t_p).max())
        hz = max(np.abs(x).max(), np.abs(u).max())
        tt = max(np.abs(t_s).max(), np.abs(t_z).max(), np.abs(t_p).max())
        rho[nu] = res
        rho_rel[nu] = res / (1.0 + max(hz, tt))
        th = theta[nu + 1]
        if nu == 0:
            xbar, ubar = x.copy(), u.copy()
        else:
            xbar = (1.0 - th) * xbar + th * x
            ubar = (1.0 - th) * ubar + th * u
        if tol is not None and rho_rel[nu] <= tol:
            rho, rho_rel = rho[:nu + 1], rho_rel[:nu + 1]
            break
    return SimpleNamespace(x=x, u=u, t_s=t_s, t_z=t_z, t_p=t_p,
                           y=(y_s, y_z, y_p), y_prev=(yp_s, yp_z, yp_p),
                           rho=rho, rho_rel=rho_rel, xbar=xbar, ubar=ubar, theta=theta)
