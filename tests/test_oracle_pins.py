"""Pins of the FP64 oracle against things other than itself.

Each check is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign, a transposed operand, the misprinted beta of App. A) makes it fail;
``test_pins_catch_planted_mistakes`` plants such slips in copies of the oracle's
data and asserts that the pins notice them.
"""
from types import SimpleNamespace

import numpy as np
import pytest

import synth
from oracle import (Tree, apg, cost_update, dense_dual_hessian, factor, jacobi_steps,
                    lipschitz_dense, prox_box, prox_dist, prox_g, solve_step, theta_sequence)
from tests import dense_reference as dr


def build(P):
    tree = Tree(P["tree"]["parent"], P["tree"]["prob"])
    fac = factor(P["net"], P["cost"])
    cu = cost_update(fac, P["cost"], tree, P["alpha2"], P["dhat"], P["eps"], P["q"])
    return tree, fac, cu


def rand_w(rng, tree, fac, scale=1.0):
    return (scale * rng.standard_normal((tree.n, fac.n_x)), scale * rng.standard_normal((tree.n, fac.n_x)),
            scale * rng.standard_normal((tree.n, fac.n_u)))


def relerr(a, b):
    return np.abs(a - b).max() / (1.0 + np.abs(b).max())


INSTANCES = [lambda: synth.tiny(0), lambda: synth.random_instance(1), lambda: synth.random_instance(2),
             lambda: synth.custom(3, 2, 4, 2, 1, synth.make_tree([1], 6))]
# a general state matrix (App. B: q_n = A' s_n in the backward sweep, x_n = A x_parent + ... forward)
GENERAL_A = [lambda: synth.general_dynamics(synth.tiny(0)), lambda: synth.general_dynamics(synth.random_instance(2), 1)]


# ---------------------------------------------------------------- prox (App. C)
def brute_prox_dist(v, P, gm):
    """1-D brute force: the prox of gm * dist(.|C) lies on the segment [v, P(v)]."""
    s = np.linspace(0.0, 1.0, 200001)
    pts = v[None, :] + s[:, None] * (P - v)[None, :]
    dist_to_C = (1.0 - s) * np.linalg.norm(P - v)            # P(pts) = P on that segment
    obj = gm * dist_to_C + 0.5 * np.sum((pts - v[None, :]) ** 2, axis=1)
    return pts[np.argmin(obj)]


@pytest.mark.parametrize("seed", range(6))
def test_prox_dist_matches_bruteforce(seed):
    rng = np.random.default_rng(seed)
    lo, hi = rng.uniform(-1, 0, 4), rng.uniform(0.5, 2, 4)
    v = rng.uniform(-4, 4, 4)
    P = prox_box(v, lo, hi)
    for gm in (0.01, 0.5, 2.0, 50.0):
        got = prox_dist(v[None, :], P[None, :], gm)[0]
        ref = brute_prox_dist(v, P, gm)
        assert np.abs(got - ref).max() < 1e-4 * (1 + np.linalg.norm(v))


def test_prox_moreau_identity():
    # prox_{g}(v) + prox_{g*}(v) = v with g = mu dist_C and g* = indicator of the mu-ball
    # plus the support function of C; on the safety set the conjugate prox is the
    # projection of v - P_C(v) onto the mu-ball when v - P_C(v) is the normal part.
    rng = np.random.default_rng(7)
    xs = rng.uniform(0, 1, 5)
    for _ in range(20):
        v = rng.uniform(-3, 3, 5)
        P = np.maximum(v, xs)
        mu = rng.uniform(0.1, 3)
        t = prox_dist(v[None, :], P[None, :], mu)[0]
        r = v - P
        nr = np.linalg.norm(r)
        y = r if nr <= mu else mu * r / nr                     # projection onto the mu-ball
        assert np.abs(t + y - v).max() < 1e-12


# ---------------------------------------------------------------- theta recursion
def test_theta_identity_and_rate():
    th = theta_sequence(2000)
    for nu in range(1, len(th) - 1):
        a, b = th[nu], th[nu + 1]
        assert abs((1 - b) / b ** 2 - 1 / a ** 2) <= 1e-12 / a ** 2
    nu = np.arange(1, 2001)
    assert np.all(np.abs(th[2:] * (nu + 2) - 2) < 0.5)
    assert abs(th[-1] * 2002 - 2) < 0.01


# ---------------------------------------------------------------- factor and cost update (App. A, B)
@pytest.mark.parametrize("mk", INSTANCES)
def test_factor_identities(mk):
    P = mk()
    tree, fac, cu = build(P)
    n_v = fac.n_v
    assert np.abs(P["net"]["E"] @ fac.L).max() <= 1e-13 * max(1, np.abs(P["net"]["E"]).max())
    assert np.abs(fac.L.T @ fac.L - np.eye(n_v)).max() < 1e-13
    assert np.linalg.eigvalsh(fac.R_bar).min() > 0
    assert np.abs(fac.Lam @ fac.R_bar + np.eye(n_v)).max() < 1e-10
    assert np.abs(fac.Phi - fac.Lam @ fac.B_bar.T).max() < 1e-12 * (1 + np.abs(fac.Phi).max())
    assert np.abs(fac.Psi - fac.Lam @ fac.L.T).max() < 1e-12 * (1 + np.abs(fac.Psi).max())
    # u_hat satisfies the coupling at every node (eq. new:decision)
    d = dr.demands(P)
    assert np.abs(cu.u_hat @ P["net"]["E"].T + d @ P["net"]["Ed"].T).max() < 1e-12


def v_form(P, tree, fac, cu, v):
    """eq. new:stage:cost: sum p_bar v'R_bar v - 2 p v_pi' R_bar v + beta' v."""
    val = 0.0
    for m in range(tree.n):
        vp = v[tree.parent[m]] if tree.parent[m] >= 0 else np.zeros(fac.n_v)
        val += cu.p_bar[m] * v[m] @ fac.R_bar @ v[m] - 2 * tree.prob[m] * vp @ fac.R_bar @ v[m] + cu.beta[m] @ v[m]
    return val


def u_form(P, tree, fac, cu, v):
    """sum p [l^w(u) + l^Delta(Delta u)] with u = L v + u_hat (eq. cost:temp, original form)."""
    c = P["cost"]
    u = v @ fac.L.T + cu.u_hat
    val = 0.0
    for m in range(tree.n):
        up = u[tree.parent[m]] if tree.parent[m] >= 0 else P["q"]
        du = u[m] - up
        val += tree.prob[m] * (c["W_alpha"] * (c["alpha1"] + P["alpha2"][tree.stage[m]]) @ u[m] + du @ c["W_u"] @ du)
    return val


def beta_gap(P, tree, fac, cu, seed=0):
    rng = np.random.default_rng(seed)
    gaps = [u_form(P, tree, fac, cu, v) - v_form(P, tree, fac, cu, v)
            for v in (rng.standard_normal((tree.n, fac.n_v)) for _ in range(4))]
    return max(gaps) - min(gaps), max(abs(g) for g in gaps)


@pytest.mark.parametrize("mk", INSTANCES)
def test_beta_by_cost_expansion(mk):
    # u-form minus v-form must not depend on v (eq. new:stage:cost expands eq. cost:delta)
    P = mk()
    tree, fac, cu = build(P)
    spread, scale = beta_gap(P, tree, fac, cu)
    assert spread < 1e-9 * (1 + scale)


# ---------------------------------------------------------------- Algorithm 1 vs dense KKT
@pytest.mark.parametrize("mk", INSTANCES + GENERAL_A)
def test_solve_step_equals_dense_kkt(mk):
    P = mk()
    tree, fac, cu = build(P)
    rng = np.random.default_rng(11)
    for scale in (0.0, 1.0, 100.0):
        w = rand_w(rng, tree, fac, scale)
        x, u = solve_step(fac, tree, cu, *w, P["p"])
        xr, ur = dr.kkt_solve(P, w)
        assert relerr(x, xr) < 1e-10 and relerr(u, ur) < 1e-10


def test_reduced_form_equals_three_term_form():
    # delta_n = (Phi s + Psi psi + Lambda sigma)/(2p) = Lambda r_n / (2 p_n) with r_n as in Algorithm 1
    P = synth.random_instance(5)
    tree, fac, cu = build(P)
    w = rand_w(np.random.default_rng(3), tree, fac)
    _, _, inn = solve_step(fac, tree, cu, *w, P["p"], return_internals=True)
    red = inn["r"] @ fac.Lam.T / (2 * tree.prob)[:, None]
    assert relerr(red, inn["delta"]) < 1e-12


@pytest.mark.parametrize("mk", INSTANCES + GENERAL_A)
def test_invariants_dynamics_coupling_nonanticipativity(mk):
    P = mk()
    tree, fac, cu = build(P)
    w = rand_w(np.random.default_rng(5), tree, fac, 10.0)
    x, u = solve_step(fac, tree, cu, *w, P["p"])
    net = P["net"]
    d = dr.demands(P)
    xpar = np.where(tree.parent[:, None] >= 0, x[np.maximum(tree.parent, 0)], P["p"][None, :])
    dyn = x - xpar @ net["A"].T - u @ net["B"].T - d @ net["Gd"].T
    assert np.abs(dyn).max() < 1e-12 * (1 + np.abs(x).max())
    assert np.abs(u @ net["E"].T + d @ net["Ed"].T).max() < 1e-12 * (1 + np.abs(u).max())
    # non-anticipativity: scenarios sharing the path to stage j share u up to stage j
    paths = tree.scenario_paths()
    U = [np.stack([u[m] for m in pth]) for pth in paths]
    for a in range(len(paths)):
        for b in range(a + 1, len(paths)):
            k = 0
            while k < len(paths[a]) and paths[a][k] == paths[b][k]:
                assert np.array_equal(U[a][k], U[b][k])
                k += 1


def test_special_case_zero_dual_constant_uhat():
    # w = 0, alpha = 0, constant demand at every node and q = u_hat: beta = 0, so delta = 0 and u = u_hat
    P = synth.random_instance(6)
    P["cost"]["alpha1"] = np.zeros_like(P["cost"]["alpha1"])
    P["alpha2"] = np.zeros_like(P["alpha2"])
    P["dhat"] = np.repeat(P["dhat"][:1], P["dhat"].shape[0], 0)
    P["eps"] = np.zeros_like(P["eps"])
    tree, fac, _ = build(P)
    d0 = P["dhat"][0]
    P["q"] = fac.P_u @ d0
    cu = cost_update(fac, P["cost"], tree, P["alpha2"], P["dhat"], P["eps"], P["q"])
    assert np.abs(cu.beta).max() < 1e-12
    z = (np.zeros((tree.n, fac.n_x)), np.zeros((tree.n, fac.n_x)), np.zeros((tree.n, fac.n_u)))
    x, u, inn = solve_step(fac, tree, cu, *z, P["p"], return_internals=True)
    assert np.abs(inn["delta"]).max() < 1e-12
    assert np.abs(u - cu.u_hat).max() < 1e-12


def test_scalar_system_by_hand():
    # n_x = n_u = n_v = 1, no coupling, chain of 2 nodes, p = 1: minimise
    # w_u (u0 - q)^2 + w_u (u1 - u0)^2 + a (u0 + u1) + xi0 x0 + xi1 x1 + psi0 u0 + psi1 u1
    # with x0 = p0 + b u0 + g d0, x1 = x0 + b u1 + g d1 (A = 1).
    b_, g_, wu, a = 2.0, -1.0, 3.0, 0.5
    P = {"net": {"n_x": 1, "n_u": 1, "n_d": 1, "n_e": 0, "A": np.eye(1), "B": np.array([[b_]]),
                 "Gd": np.array([[g_]]), "E": np.zeros((0, 1)), "Ed": np.zeros((0, 1))},
         "cost": {"W_alpha": 1.0, "alpha1": np.array([a]), "W_u": np.array([[wu]]), "W_x": 1.0, "gamma_d": 1.0},
         "tree": {"parent": np.array([-1, 0]), "prob": np.array([1.0, 1.0]), "stage": np.array([0, 1])},
         "alpha2": np.zeros((2, 1)), "p": np.array([1.0]), "q": np.array([0.4]),
         "dhat": np.array([[0.3], [0.7]]), "eps": np.zeros((2, 1))}
    tree, fac, cu = build(P)
    xi = np.array([[0.2], [-0.1]]); psi = np.array([[0.05], [0.3]])
    x, u = solve_step(fac, tree, cu, xi, np.zeros((2, 1)), psi, P["p"])
    # stationarity in (u0, u1), x eliminated: hand-derived 2x2 system
    # d/du0: 2wu(u0-q) - 2wu(u1-u0) + a + psi0 + b(xi0 + xi1) = 0
    # d/du1: 2wu(u1-u0) + a + psi1 + b xi1 = 0
    K = np.array([[4 * wu, -2 * wu], [-2 * wu, 2 * wu]])
    rhs = np.array([2 * wu * 0.4 - a - psi[0, 0] - b_ * (xi[0, 0] + xi[1, 0]), -a - psi[1, 0] - b_ * xi[1, 0]])
    uu = np.linalg.solve(K, rhs)
    assert np.abs(u[:, 0] - uu).max() < 1e-13
    x0 = 1.0 + b_ * uu[0] + g_ * 0.3
    assert abs(x[0, 0] - x0) < 1e-13 and abs(x[1, 0] - (x0 + b_ * uu[1] + g_ * 0.7)) < 1e-13


# ---------------------------------------------------------------- dual Hessian (Sec. IV-D)
def closed_form_diagonal(fac, tree):
    """Hand derivation for A = I: the response of x_n to xi_n sums, over ancestors a
    of n (and n), k_a^2/(2 p_a) B_bar R_bar^{-1} B_bar' with k_a the number of path
    nodes from a down to n; the response of u_n to psi_n sums 1/(2 p_a) L R_bar^{-1} L'."""
    Rinv = np.linalg.inv(fac.R_bar)
    dB = np.einsum("ij,jk,ik->i", fac.B_bar, Rinv, fac.B_bar)
    dL = np.einsum("ij,jk,ik->i", fac.L, Rinv, fac.L)
    cx, cu_ = np.zeros(tree.n), np.zeros(tree.n)
    for m in range(tree.n):
        path = tree.path(m)
        for i, a in enumerate(path):
            k = len(path) - i
            cx[m] += k * k / (2 * tree.prob[a])
            cu_[m] += 1.0 / (2 * tree.prob[a])
    return cx[:, None] * dB[None, :], cu_[:, None] * dL[None, :]


@pytest.mark.parametrize("mk", INSTANCES[:3])
def test_dense_dual_hessian(mk):
    P = mk()
    tree, fac, cu = build(P)
    M = dense_dual_hessian(fac, tree)
    assert np.abs(M - M.T).max() < 1e-10 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > -1e-9 * np.abs(M).max()
    dx, du = closed_form_diagonal(fac, tree)
    blk = 2 * fac.n_x + fac.n_u
    dg = np.diag(M).reshape(tree.n, blk)
    assert relerr(dg[:, :fac.n_x], dx) < 1e-12
    assert relerr(dg[:, fac.n_x:2 * fac.n_x], dx) < 1e-12
    assert relerr(dg[:, 2 * fac.n_x:], du) < 1e-12
    # the Hessian is the linear part of w -> -H z(w), also available from the dense KKT
    rng = np.random.default_rng(2)
    w = rand_w(rng, tree, fac)
    x0, u0 = dr.kkt_solve(P, tuple(np.zeros_like(a) for a in w))
    x1, u1 = dr.kkt_solve(P, w)
    Mw = M @ np.concatenate([w[0], w[1], w[2]], axis=1).ravel()
    ref = -np.concatenate([x1 - x0, x1 - x0, u1 - u0], axis=1).ravel()
    assert relerr(Mw, ref) < 1e-9


# ---------------------------------------------------------------- converged APG
def micro_instance(seed):
    return synth.custom(seed, n_x=1, n_u=2, n_d=1, n_e=1, tree=synth.make_tree([2], 2),
                        weights=(1.0, 1.0, 4.0, 20.0))


@pytest.mark.parametrize("seed,a", [(0, None), (1, None), (2, None), (3, 0.9)])
def test_apg_converges_to_bruteforce_optimum(seed, a):
    P = micro_instance(seed)
    if a is not None:  # a leaking tank: x+ = a x + B u + G d
        P["net"] = {**P["net"], "A": np.array([[a]])}
    # push the states against their bounds so several pieces are active
    P["p"] = np.array([2.0 + seed])
    tree, fac, cu = build(P)
    best = dr.active_set_bruteforce(P)
    assert best is not None
    steps = jacobi_steps(fac, tree)
    R = apg(fac, tree, cu, P["cost"], P["p"], steps, 20000)
    assert np.abs(R.u - best[2]).max() < 1e-6 * (1 + np.abs(best[2]).max())
    assert np.abs(R.x - best[1]).max() < 1e-6 * (1 + np.abs(best[1]).max())
    assert abs(dr.objective(P, R.x, R.u) - best[0]) < 1e-7 * (1 + abs(best[0]))


def test_apg_optimality_certificate_tiny():
    """Converged APG output satisfies the optimality conditions of the problem:
    z = argmin f + <Hz, y> (dense KKT) and y in the subdifferential of g at Hz."""
    P = synth.tiny(0)
    tree, fac, cu = build(P)
    steps = jacobi_steps(fac, tree)
    R = apg(fac, tree, cu, P["cost"], P["p"], steps, 6000)
    assert R.rho_rel[-1] < 1e-5
    c = P["cost"]
    y_s, y_z, y_p = R.y
    x, u = R.x, R.u
    xr, ur = dr.kkt_solve(P, R.y)
    assert relerr(x, xr) < 1e-4 and relerr(u, ur) < 1e-4
    tol = 1e-4
    ysc = 1 + np.abs(y_p).max()
    for m in range(tree.n):
        for i in range(fac.n_u):
            if y_p[m, i] > tol * ysc:
                assert u[m, i] > c["u_max"][i] - 1e-3
            if y_p[m, i] < -tol * ysc:
                assert u[m, i] < c["u_min"][i] + 1e-3
        for yb, lo, hi, mu in ((y_s[m], c["x_s"], np.full(fac.n_x, np.inf), tree.prob[m] * c["W_x"]),
                               (y_z[m], c["x_min"], c["x_max"], c["gamma_d"])):
            r = x[m] - np.clip(x[m], lo, hi)
            assert np.linalg.norm(yb) <= mu * (1 + 1e-6) + 1e-9
            if np.linalg.norm(r) > 1e-3:
                assert np.abs(yb - mu * r / np.linalg.norm(r)).max() < 1e-3 * mu
            else:          # normal cone of C at x: zero on strictly inactive entries, outward sign elsewhere
                inner = (x[m] > lo + 1e-3) & (x[m] < hi - 1e-3)
                assert np.abs(yb[inner]).max(initial=0.0) < 1e-3 * mu
                assert np.all(yb[x[m] <= lo + 1e-3] <= 1e-3 * mu)
                assert np.all(yb[x[m] >= hi - 1e-3] >= -1e-3 * mu)


def test_jacobi_lipschitz_bounds_step():
    P = synth.tiny(0)
    tree, fac, cu = build(P)
    M = dense_dual_hessian(fac, tree)
    L = lipschitz_dense(M)
    v = np.random.default_rng(0).standard_normal(M.shape[0])
    assert v @ M @ v <= L * (v @ v) * (1 + 1e-12)
    st = jacobi_steps(fac, tree, M)
    assert st["lambda"] > 0


def kkt_dual_hessian(P):
    """The dual Hessian column by column from the dense KKT solve of the whole problem
    (independent of Algorithm 1): column k is -(Hz(e_k) - Hz(0))."""
    tree = P["tree"]
    n, n_x, n_u = len(tree["parent"]), P["net"]["n_x"], P["net"]["n_u"]
    blk = 2 * n_x + n_u
    zero = (np.zeros((n, n_x)), np.zeros((n, n_x)), np.zeros((n, n_u)))
    x0, u0 = dr.kkt_solve(P, zero)
    M = np.zeros((n * blk, n * blk))
    for k in range(n * blk):
        w = np.zeros((n, blk))
        w.flat[k] = 1.0
        x1, u1 = dr.kkt_solve(P, (w[:, :n_x], w[:, n_x:2 * n_x], w[:, 2 * n_x:]))
        M[:, k] = -np.concatenate([x1 - x0, x1 - x0, u1 - u0], axis=1).ravel()
    return M


@pytest.mark.parametrize("mk", INSTANCES)
def test_jacobi_steps_from_the_hand_diagonal(mk):
    """Sec. IV-D reading: one scalar 1/mean(diag) per distance block, 1/diag per input entry
    (an entry of zero curvature takes the mean of its node's other entries), and
    lambda = 1 / largest eigenvalue of the scaled dual Hessian.  The diagonal comes from
    the hand derivation for A = I and the eigenvalue from the dense KKT Hessian."""
    P = mk()
    tree, fac, cu = build(P)
    st = jacobi_steps(fac, tree)
    dx, du = closed_form_diagonal(fac, tree)
    d_s = 1.0 / dx.mean(axis=1)
    live = du > 1e-12 * du.max(axis=1, keepdims=True)
    d_p = np.empty_like(du)
    for m in range(tree.n):
        fill = du[m, live[m]].mean()
        d_p[m] = 1.0 / np.where(live[m], du[m], fill)
    assert relerr(st["d_s"], d_s) < 1e-12 and relerr(st["d_z"], d_s) < 1e-12
    assert relerr(st["d_p"], d_p) < 1e-12
    dvec = np.concatenate([np.repeat(d_s[:, None], fac.n_x, 1), np.repeat(d_s[:, None], fac.n_x, 1), d_p],
                          axis=1).ravel()
    M = kkt_dual_hessian(P)
    sq = np.sqrt(dvec)
    lam = 1.0 / np.linalg.eigvalsh(sq[:, None] * M * sq[None, :]).max()
    assert abs(st["lambda"] - lam) < 1e-9 * lam
    assert relerr(st["s"], lam * d_s) < 1e-9 and relerr(st["p"], lam * d_p) < 1e-9


def test_ergodic_average_is_the_theta_weighted_mean():
    """Sec. IV-A: zbar^nu = (1 - theta_nu) zbar^{nu-1} + theta_nu z^nu with theta_0 = 1.  Since
    (1 - theta_nu) / theta_nu^2 = 1 / theta_{nu-1}^2, unrolling gives the closed form
    zbar^nu = theta_nu^2 sum_k z^k / theta_k, a convex combination (the weights telescope to
    one), so zbar also meets the dynamics and the coupling."""
    P = synth.random_instance(2)
    tree, fac, cu = build(P)
    steps = jacobi_steps(fac, tree)
    K = 12
    xs, us = [], []
    for k in range(1, K + 1):               # z^{k-1} is the last primal iterate of a k-iteration run
        Rk = apg(fac, tree, cu, P["cost"], P["p"], steps, k)
        xs.append(Rk.x)
        us.append(Rk.u)
    R = apg(fac, tree, cu, P["cost"], P["p"], steps, K)
    th = 1.0
    thetas = [th]
    for _ in range(K - 1):
        th = 0.5 * th * (np.sqrt(th * th + 4.0) - th)
        thetas.append(th)
    wts = np.array([thetas[-1] ** 2 / t for t in thetas])
    assert abs(wts.sum() - 1.0) < 1e-12
    xbar = sum(wk * xk for wk, xk in zip(wts, xs))
    ubar = sum(wk * uk for wk, uk in zip(wts, us))
    assert relerr(R.xbar, xbar) < 1e-12 and relerr(R.ubar, ubar) < 1e-12
    assert relerr(R.xbar, xs[-1]) > 1e-6                     # the average is not the last iterate
    net = P["net"]
    d = dr.demands(P)
    xpar = np.where(tree.parent[:, None] >= 0, R.xbar[np.maximum(tree.parent, 0)], P["p"][None, :])
    dyn = R.xbar - xpar @ net["A"].T - R.ubar @ net["B"].T - d @ net["Gd"].T
    assert np.abs(dyn).max() < 1e-11 * (1 + np.abs(R.xbar).max())
    assert np.abs(R.ubar @ net["E"].T + d @ net["Ed"].T).max() < 1e-11 * (1 + np.abs(R.ubar).max())


# ---------------------------------------------------------------- the pins notice planted mistakes
# ---------------------------------------------------------------- dual rate (Sec. IV-A)
def dual_value(P, y, mu_s):
    """D(y) = min_z f(z) + <y, H z> - g*(y), with z(y) from the dense KKT solve and the
    conjugates of the three blocks of g: <y, x_s> on y <= 0 with ||y|| <= mu_S (safety
    distance to {x >= x_s}), the support function of [x_min, x_max] with ||y|| <= gamma_d,
    and the support function of [u_min, u_max] (input box).  Also returns how far y is
    from the domain of g* (0 inside)."""
    cost, tree = P["cost"], P["tree"]
    ys, yz, yp = y
    x, u = dr.kkt_solve(P, y)
    Q, c, _, _ = dr.quadratic_data(P)
    z = np.concatenate([x.ravel(), u.ravel()])
    f = 0.5 * z @ Q @ z + c @ z + tree["prob"][0] * P["q"] @ cost["W_u"] @ P["q"]
    lin = np.sum(ys * x) + np.sum(yz * x) + np.sum(yp * u)
    gs = np.sum(ys * cost["x_s"])
    gz = np.sum(np.maximum(yz * cost["x_min"], yz * cost["x_max"]))
    gp = np.sum(np.maximum(yp * cost["u_min"], yp * cost["u_max"]))
    out = max(ys.max(), (np.linalg.norm(ys, axis=1) / mu_s).max() - 1.0,
              (np.linalg.norm(yz, axis=1) / cost["gamma_d"]).max() - 1.0, 0.0)
    return f + lin - gs - gz - gp, out


def _dual_rate_setup(P):
    tree, fac, cu = build(P)
    M = dense_dual_hessian(fac, tree)
    L = np.linalg.eigvalsh(0.5 * (M + M.T)).max()
    return tree, fac, cu, L, tree.prob * P["cost"]["W_x"]


@pytest.mark.parametrize("mk", INSTANCES[:2] + GENERAL_A[:1])
def test_apg_dual_rate_and_zero_duality_gap(mk):
    """With the scalar step 1/L_D the iteration is the accelerated proximal gradient method
    on the dual: D* - D(y^nu) <= 2 L_D ||y^0 - y*||^2 / (nu + 1)^2.  Every iterate lies in
    the domain of g*, and at the solution the dual value meets the primal objective."""
    P = mk()
    tree, fac, cu, L, mu_s = _dual_rate_setup(P)
    R = apg(fac, tree, cu, P["cost"], P["p"], 1.0 / L, 20000)
    d_star, out = dual_value(P, R.y, mu_s)
    assert out < 1e-12
    primal = dr.objective(P, R.x, R.u, mu_s)
    assert abs(primal - d_star) <= 1e-4 * (1 + abs(d_star))       # strong duality
    r2 = sum(np.sum(a ** 2) for a in R.y)                          # y^0 = 0
    for nu in (5, 20, 80, 320, 1280):
        Rn = apg(fac, tree, cu, P["cost"], P["p"], 1.0 / L, nu)
        d, out = dual_value(P, Rn.y, mu_s)
        assert out < 1e-12, nu
        assert d <= primal + 1e-9 * (1 + abs(primal)), nu          # weak duality
        assert d_star - d <= 2 * L * r2 / (nu + 1) ** 2, nu


def test_pins_catch_planted_mistakes():
    P = synth.random_instance(2)         # branching tree: probabilities below one
    tree, fac, cu = build(P)
    w = rand_w(np.random.default_rng(9), tree, fac, 3.0)
    xr, ur = dr.kkt_solve(P, w)

    def kkt_err(f, c):
        x, u = solve_step(f, tree, c, *w, P["p"])
        return max(relerr(x, xr), relerr(u, ur))

    assert kkt_err(fac, cu) < 1e-10
    # printed eq. appendix:beta: extra p_n on the R_hat term and no p_n on u_hat_pi
    d = dr.demands(P)
    u_hat = cu.u_hat
    u_par = np.vstack([P["q"][None, :], u_hat[tree.parent[1:]]])
    child = np.zeros_like(u_hat)
    for m in range(1, tree.n):
        child[tree.parent[m]] += tree.prob[m] * u_hat[m]
    p = tree.prob[:, None]
    printed = p * cu.alpha_bar[tree.stage] + 2 * p * ((cu.p_bar[:, None] * u_hat - u_par - child) @ fac.R_hat)
    assert kkt_err(fac, SimpleNamespace(**{**vars(cu), "beta": printed})) > 1e-6
    assert beta_gap(P, tree, fac, SimpleNamespace(**{**vars(cu), "beta": printed}))[0] > 1e-6
    # sign of Lambda flipped
    bad = SimpleNamespace(**{**vars(fac), "Lam": -fac.Lam})
    assert kkt_err(bad, cu) > 1e-6
    # the Psi term dropped
    bad = SimpleNamespace(**{**vars(fac), "Psi": 0 * fac.Psi})
    assert kkt_err(bad, cu) > 1e-6
    # u_{-1} = q forgotten (u_hat_pi(root) = 0)
    cu0 = cost_update(fac, P["cost"], tree, P["alpha2"], P["dhat"], P["eps"], 0 * P["q"])
    assert kkt_err(fac, cu0) > 1e-6
    # e without the demand term
    bad = SimpleNamespace(**{**vars(cu), "e": u_hat @ P["net"]["B"].T})
    assert kkt_err(fac, bad) > 1e-6
    # prox without the gamma*mu factor in the far branch fails the brute-force prox
    v = np.array([3.0, -2.0, 0.5]); Pv = np.maximum(v, 1.0); gm = 0.7
    far = v + (Pv - v) / np.linalg.norm(Pv - v)
    assert np.abs(far - brute_prox_dist(v, Pv, gm)).max() > 1e-3
    # the extrapolation dropped (plain proximal gradient on the dual) breaks the O(1/nu^2) bound
    Pt = synth.tiny(0)
    tree_t, fac_t, cu_t, L, mu_t = _dual_rate_setup(Pt)
    R = apg(fac_t, tree_t, cu_t, Pt["cost"], Pt["p"], 1.0 / L, 20000)
    d_star = dual_value(Pt, R.y, mu_t)[0]
    r2 = sum(np.sum(a ** 2) for a in R.y)
    lam, n = 1.0 / L, tree_t.n
    y = [np.zeros((n, fac_t.n_x)), np.zeros((n, fac_t.n_x)), np.zeros((n, fac_t.n_u))]
    nu = 320
    for _ in range(nu):
        x, u = solve_step(fac_t, tree_t, cu_t, *y, Pt["p"])
        t_s, t_z, t_p = prox_g(y[0] / lam + x, y[1] / lam + x, y[2] / lam + u, Pt["cost"], mu_t,
                               np.full(n, lam), np.full(n, lam))
        y = [y[0] + lam * (x - t_s), y[1] + lam * (x - t_z), y[2] + lam * (u - t_p)]
    assert d_star - dual_value(Pt, y, mu_t)[0] > 2 * L * r2 / (nu + 1) ** 2
    # with a general A, an oracle that drops A (q_n = s_n, x_n = x_parent + ...) fails the dense KKT
    Pa = synth.general_dynamics(synth.random_instance(2), 1)
    tree_a, fac_a, cu_a = build(Pa)
    wa = rand_w(np.random.default_rng(4), tree_a, fac_a, 3.0)
    xr_a, ur_a = dr.kkt_solve(Pa, wa)
    x_ok, u_ok = solve_step(fac_a, tree_a, cu_a, *wa, Pa["p"])
    assert max(relerr(x_ok, xr_a), relerr(u_ok, ur_a)) < 1e-10
    no_a = SimpleNamespace(**{**vars(fac_a), "A": np.eye(fac_a.n_x)})
    x_bad, u_bad = solve_step(no_a, tree_a, cu_a, *wa, Pa["p"])
    assert max(relerr(x_bad, xr_a), relerr(u_bad, ur_a)) > 1e-6
    # theta with the wrong sign fails the identity
    a = 0.5
    b = 0.5 * (np.sqrt(a ** 4 + 4 * a ** 2) + a ** 2)
    assert abs((1 - b) / b ** 2 - 1 / a ** 2) > 1e-3
