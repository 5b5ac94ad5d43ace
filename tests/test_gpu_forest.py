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


@pytest.mark.parametrize("schedule", [1, 2, 3])
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
    members, F, steps, per = _forest_case(4, 4)
    g = H.Gpu(F, steps=steps, precision=precision, shared_packs=1)
    try:
        info = g.solve(300)
    finally:
        g.close()
    g64 = H.Gpu(F, steps=steps, precision=0, shared_packs=1)
    try:
        ref = g64.solve(300)
    finally:
        g64.close()
    assert abs(info["rho_rel"] - ref["rho_rel"]) <= 1e-4
