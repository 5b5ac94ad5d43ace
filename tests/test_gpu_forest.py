"""Batching: a forest of uneven trees on one network, solved by one set of launches
per iteration, gives every member tree the iterates of the FP64 oracle run on that
tree alone (the trees share nothing but the iteration count and the theta sequence)."""
import numpy as np
import pytest

import oracle
import synth
from tests import harness as H

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-9


def _forest_case(seed, count):
    members = synth.forest_members(seed, count, max_horizon=7)
    F = synth.forest(members)
    n = len(F["tree"]["parent"])
    n_u = F["net"]["n_u"]
    steps = {"s": np.zeros(n), "z": np.zeros(n), "p": np.zeros((n, n_u))}
    per = []
    for r, P in enumerate(members):
        tree, fac, _ = H.oracle_build(P)
        st = oracle.jacobi_steps(fac, tree)
        idx = F["members"][r]
        for k in ("s", "z", "p"):
            steps[k][idx] = st[k]
        per.append(st)
    return members, F, steps, per


@pytest.mark.parametrize("schedule", [1, 2, 3, 4])
@pytest.mark.parametrize("shared", [0, 1])
def test_forest_matches_each_tree_alone(schedule, shared):
    members, F, steps, per = _forest_case(0, 5)
    iters = 120
    g = H.Gpu(F, steps=steps, schedule=schedule, shared_packs=shared)
    try:
        info = g.solve(iters)
        u, x, y = g.arrays()
        assert g.smpc.smpc_tree_info_get(g.tree)["n_trees"] == len(members)
    finally:
        g.close()
    rho = 0.0
    n_u = F["net"]["n_u"]
    for r, P in enumerate(members):
        R = H.oracle_run(P, per[r], iters)
        idx = F["members"][r]
        e = (H.relerr(u[idx], R.u), H.relerr(x[idx], R.x), H.relerr(y[idx], H.stack_y(R.y)))
        assert max(e) <= FP64_TOL, (r, e)
        assert np.abs(info["u0"][r * n_u:(r + 1) * n_u] - R.u[0]).max() <= FP64_TOL * (1 + np.abs(R.u[0]).max())
        rho = max(rho, R.rho[-1])
    assert abs(info["rho"] - rho) <= FP64_TOL * (1 + rho) * 10


@pytest.mark.parametrize("precision", [1, 2])
def test_forest_reduced_precision(precision):
    """Every member tree of a float32 / bfloat16 forest against the FP64 oracle run on that
    tree alone, with the bars of the full-size reduced-precision tests at equal iteration
    counts: float32 1e-4 elementwise (relative to 1 + the largest entry) and |rho_rel| of
    each tree within 1e-4; bfloat16 (anchored) 0.15 and 0.05."""
    members, F, steps, per = _forest_case(4, 4)
    iters = 300
    g = H.Gpu(F, steps=steps, precision=precision, shared_packs=1)
    try:
        g.solve(iters)
        u, x, y = g.arrays()
        its, rr = g.smpc.smpc_solve_trees(g.fac, len(members))
    finally:
        g.close()
    bound, rho_bound = {1: (1e-4, 1e-4), 2: (0.15, 0.05)}[precision]
    for r, P in enumerate(members):
        R = H.oracle_run(P, per[r], iters)
        idx = F["members"][r]
        e = (H.relerr(u[idx], R.u), H.relerr(x[idx], R.x), H.relerr(y[idx], H.stack_y(R.y)))
        assert max(e) <= bound, (r, e)
        assert its[r] == iters
        assert abs(rr[r] - R.rho_rel[-1]) <= rho_bound, (r, rr[r], R.rho_rel[-1])


@pytest.mark.parametrize("schedule", [1, 2, 3, 4])
@pytest.mark.parametrize("shared", [0, 1])
def test_forest_stops_each_tree_on_its_own(schedule, shared):
    """With a tolerance, every tree of a forest stops at its own first iterate whose relative
    residual (over that tree's nodes, Sec. IV-E) meets it, exactly as the oracle stops on
    that tree alone; the stopped tree keeps that iterate while the others go on."""
    members, F, steps, per = _forest_case(7, 5)
    tol, cap = 2e-4, 4000
    g = H.Gpu(F, steps=steps, schedule=schedule, shared_packs=shared)
    try:
        info = g.solve(cap, tol=tol, check_every=32)
        u, x, y = g.arrays()
        its, rr = g.smpc.smpc_solve_trees(g.fac, len(members))
    finally:
        g.close()
    counts = []
    for r, P in enumerate(members):
        tree, fac, cu = H.oracle_build(P)
        R = oracle.apg(fac, tree, cu, P["cost"], P["p"], per[r], cap, tol=tol)
        k = len(R.rho_rel)
        counts.append(k)
        assert R.rho_rel[-1] <= tol, r
        assert its[r] == k, (r, its[r], k)
        idx = F["members"][r]
        e = (H.relerr(u[idx], R.u), H.relerr(x[idx], R.x), H.relerr(y[idx], H.stack_y(R.y)))
        assert max(e) <= FP64_TOL, (r, e)
        assert abs(rr[r] - R.rho_rel[-1]) <= 1e-9, (r, rr[r], R.rho_rel[-1])
    assert len(set(counts)) > 1, counts  # the trees stop at different iterations
    assert info["iterations"] == max(counts)
