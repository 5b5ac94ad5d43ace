"""Independent dense restatements of the SMPC problem, used to pin the oracle.

Everything here works in the original variables z = (x_n, u_n) of the problem
statement (Sec. III-D, eq. Sc-MPC and eq. fz), without the null-space
elimination, the factor step or Algorithm 1:

* ``kkt_solve``: z(w) = argmin_z f(z) + <H z, w> as one equality-constrained
  quadratic program (dynamics and coupling as constraints) solved with a dense
  linear solve of its KKT system;
* ``objective``: the full soft-constrained objective f(z) + g(H z);
* ``active_set_bruteforce``: exact minimiser of the full problem for one-tank
  instances, by enumerating every piece of the piecewise-linear state penalties
  and every input-bound pattern and keeping the candidate whose KKT conditions hold.
"""
from __future__ import annotations

import itertools

import numpy as np


def _layout(P):
    net, tree = P["net"], P["tree"]
    n = len(tree["parent"])
    return n, net["n_x"], net["n_u"]


def demands(P):
    return P["dhat"][P["tree"]["stage"]] + P["eps"]


def quadratic_data(P, w=None):
    """0.5 z'Qz + c'z (+ const) for sum_n p_n [l^w + l^Delta] + <H z, w>, and the
    equality constraints C z = b (dynamics with x_pi(root) = p, coupling)."""
    net, cost, tree = P["net"], P["cost"], P["tree"]
    n, n_x, n_u = _layout(P)
    parent, prob, stage = tree["parent"], tree["prob"], tree["stage"]
    d = demands(P)
    nz = n * (n_x + n_u)
    xo = lambda m: m * n_x                       # noqa: E731
    uo = lambda m: n * n_x + m * n_u             # noqa: E731
    Q = np.zeros((nz, nz))
    c = np.zeros(nz)
    W = cost["W_u"]
    for m in range(n):
        pm = prob[m]
        # smoothing p_m (u_m - u_pi)' W (u_m - u_pi), u_pi(root) = q
        Q[uo(m):uo(m) + n_u, uo(m):uo(m) + n_u] += 2 * pm * W
        if parent[m] >= 0:
            a = parent[m]
            Q[uo(a):uo(a) + n_u, uo(a):uo(a) + n_u] += 2 * pm * W
            Q[uo(m):uo(m) + n_u, uo(a):uo(a) + n_u] -= 2 * pm * W
            Q[uo(a):uo(a) + n_u, uo(m):uo(m) + n_u] -= 2 * pm * W
        else:
            c[uo(m):uo(m) + n_u] += -2 * pm * W @ P["q"]
        # economic cost
        c[uo(m):uo(m) + n_u] += pm * cost["W_alpha"] * (cost["alpha1"] + P["alpha2"][stage[m]])
        if w is not None:
            ws, wz, wp = w
            c[xo(m):xo(m) + n_x] += ws[m] + wz[m]
            c[uo(m):uo(m) + n_u] += wp[m]
    n_e = net["E"].shape[0]
    C = np.zeros((n * (n_x + n_e), nz))
    b = np.zeros(n * (n_x + n_e))
    r = 0
    for m in range(n):
        C[r:r + n_x, xo(m):xo(m) + n_x] = np.eye(n_x)
        C[r:r + n_x, uo(m):uo(m) + n_u] = -net["B"]
        rhs = net["Gd"] @ d[m]
        if parent[m] >= 0:
            C[r:r + n_x, xo(parent[m]):xo(parent[m]) + n_x] = -net["A"]
        else:
            rhs = rhs + net["A"] @ P["p"]
        b[r:r + n_x] = rhs
        r += n_x
        C[r:r + n_e, uo(m):uo(m) + n_u] = net["E"]
        b[r:r + n_e] = -net["Ed"] @ d[m]
        r += n_e
    return Q, c, C, b


def split(P, z):
    n, n_x, n_u = _layout(P)
    return z[:n * n_x].reshape(n, n_x), z[n * n_x:].reshape(n, n_u)


def kkt_solve(P, w):
    Q, c, C, b = quadratic_data(P, w)
    k = C.shape[0]
    K = np.block([[Q, C.T], [C, np.zeros((k, k))]])
    sol = np.linalg.solve(K, np.concatenate([-c, b]))
    return split(P, sol[:Q.shape[0]])


def dist_box(x, lo, hi):
    return np.sqrt(np.sum((x - np.clip(x, lo, hi)) ** 2, axis=-1))


def objective(P, x, u, mu_s=None):
    cost, tree = P["cost"], P["tree"]
    Q, c, _, _ = quadratic_data(P)
    z = np.concatenate([x.ravel(), u.ravel()])
    val = 0.5 * z @ Q @ z + c @ z + tree["prob"][0] * P["q"] @ cost["W_u"] @ P["q"]
    if mu_s is None:
        mu_s = tree["prob"] * cost["W_x"]
    val += np.sum(mu_s * dist_box(x, cost["x_s"], np.inf))
    val += np.sum(cost["gamma_d"] * dist_box(x, cost["x_min"], cost["x_max"]))
    return val


def active_set_bruteforce(P, tol=1e-9):
    """Exact minimiser of f(z) + g(Hz) for n_x = 1 instances (piecewise QP)."""
    net, cost, tree = P["net"], P["cost"], P["tree"]
    n, n_x, n_u = _layout(P)
    assert n_x == 1
    Q, c, C, b = quadratic_data(P)
    nz = Q.shape[0]
    xs, lo, hi = float(cost["x_s"][0]), float(cost["x_min"][0]), float(cost["x_max"][0])
    assert lo < xs < hi
    g = cost["gamma_d"]
    mus = tree["prob"] * cost["W_x"]
    # pieces: (slope for open piece or None, breakpoint value or None, interval check)
    def pieces(mu):
        return [
            ("lt", -mu - g, None, (-np.inf, lo)), ("mid", -mu, None, (lo, xs)),
            ("ok", 0.0, None, (xs, hi)), ("gt", g, None, (hi, np.inf)),
            ("=lo", None, lo, (-mu - g, -mu)), ("=xs", None, xs, (-mu, 0.0)), ("=hi", None, hi, (0.0, g)),
        ]
    n_free = n_u - np.linalg.matrix_rank(net["E"]) if net["E"].shape[0] else n_u
    # 0 free, 1 at lower, 2 at upper; at most n_v = n_u - rank(E) entries can be pinned
    u_pats = [pt for pt in itertools.product((0, 1, 2), repeat=n_u) if sum(1 for s in pt if s) <= n_free]
    best = None
    for xsel in itertools.product(range(7), repeat=n):
        for usel in itertools.product(range(len(u_pats)), repeat=n):
            cc = c.copy()
            rows, rhs, kinds = [], [], []
            for m in range(n):
                name, slope, bp, iv = pieces(mus[m])[xsel[m]]
                if bp is None:
                    cc[m] += slope
                else:
                    e = np.zeros(nz); e[m] = 1.0
                    rows.append(e); rhs.append(bp); kinds.append(("x", m, iv))
                for i, s in enumerate(u_pats[usel[m]]):
                    if s:
                        e = np.zeros(nz); e[n + m * n_u + i] = 1.0
                        rows.append(e)
                        rhs.append(cost["u_min"][i] if s == 1 else cost["u_max"][i])
                        kinds.append(("u", (m, i), s))
            CC = np.vstack([C] + rows) if rows else C
            bb = np.concatenate([b, rhs]) if rows else b
            k = CC.shape[0]
            K = np.block([[Q, CC.T], [CC, np.zeros((k, k))]])
            try:
                sol = np.linalg.solve(K, np.concatenate([-cc, bb]))
            except np.linalg.LinAlgError:
                continue
            if np.abs(K @ sol - np.concatenate([-cc, bb])).max() > 1e-8 * (1 + np.abs(bb).max()):
                continue
            z, nu = sol[:nz], sol[nz:]
            x, u = z[:n], z[n:].reshape(n, n_u)
            ok = True
            for m in range(n):          # open pieces must hold strictly (within tol)
                name, slope, bp, iv = pieces(mus[m])[xsel[m]]
                if bp is None and not (iv[0] - tol <= x[m] <= iv[1] + tol):
                    ok = False
                    break
            if not ok:
                continue
            if np.any(u < cost["u_min"][None, :] - tol) or np.any(u > cost["u_max"][None, :] + tol):
                continue
            for j, kd in enumerate(kinds):   # multipliers of the added rows
                mult = nu[C.shape[0] + j]
                if kd[0] == "u":
                    if (kd[2] == 1 and mult > tol * (1 + abs(mult))) or (kd[2] == 2 and mult < -tol * (1 + abs(mult))):
                        ok = False
                        break
                else:                          # the row's multiplier is the subgradient used
                    a_, b_ = kd[2]
                    if not (a_ - 1e-7 * (1 + abs(a_)) <= mult <= b_ + 1e-7 * (1 + abs(b_))):
                        ok = False
                        break
            if not ok:
                continue
            val = objective(P, x.reshape(n, 1), u)
            if best is None or val < best[0] - 1e-12:
                best = (val, x.reshape(n, 1), u)
    return best
