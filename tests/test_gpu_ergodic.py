"""The ergodic primal average (Sec. IV-A, after eq. apg-iteration) through the C ABI against
the FP64 oracle's zbar, element by element: float64 at 1e-9 relative to 1 + the largest
entry (the bar of the other float64 parity tests), float32 at 1e-4, on every schedule,
with a tolerance stop, warm starts (theta restarts with every solve), forests (each tree
averages up to its own stop) and graph-captured chunks."""
import numpy as np
import pytest

import oracle
import synth
from tests import harness as H

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-9
FP32_TOL = 1e-4


def _ergodic(P, steps, iters, tol=None, y0=None):
    tree, fac, cu = H.oracle_build(P)
    return oracle.apg(fac, tree, cu, P["cost"], P["p"], steps, iters, y0=y0, tol=tol)


def _check(g, R, bound):
    ub, xb = g.bars()
    eu, ex = H.relerr(ub, R.ubar), H.relerr(xb, R.xbar)
    assert max(eu, ex) <= bound, (eu, ex)
    u, x, _ = g.arrays()
    # the average is not the last iterate (it would be for one iteration only)
    return H.relerr(ub, u), H.relerr(xb, x)


@pytest.mark.parametrize("schedule", [1, 2, 3, 4])
@pytest.mark.parametrize("name,iters", [("tiny", 1), ("tiny", 500), ("random_a", 200), ("late_branch", 200)])
def test_ergodic_average_fp64(name, iters, schedule):
    P = synth.tiny(0) if name == "tiny" else H.edge_instances()[name]
    steps = H.tiny_steps(P)
    R = _ergodic(P, steps, iters)
    g = H.Gpu(P, steps=steps, schedule=schedule)
    try:
        info = g.solve(iters, ergodic=1)
        du, dx = _check(g, R, FP64_TOL)
    finally:
        g.close()
    assert info["iterations"] == iters
    if iters > 1:
        assert max(du, dx) > 1e-6


@pytest.mark.parametrize("schedule", [2, 4])
def test_ergodic_average_full_size(schedule):
    P = synth.barcelona(0)
    steps = H.full_size_steps(P)
    iters = 60
    R = _ergodic(P, steps, iters)
    for prec, bound in ((0, FP64_TOL), (1, FP32_TOL)):
        g = H.Gpu(P, steps=steps, schedule=schedule, precision=prec)
        try:
            g.solve(iters, ergodic=1)
            _check(g, R, bound)
        finally:
            g.close()


def test_ergodic_average_with_a_tolerance_stop():
    P = synth.tiny(0)
    steps = H.tiny_steps(P)
    tol, cap = 1e-3, 5000
    R = _ergodic(P, steps, cap, tol=tol)
    g = H.Gpu(P, steps=steps)
    try:
        info = g.solve(cap, tol=tol, ergodic=1, check_every=16)
        _check(g, R, FP64_TOL)
    finally:
        g.close()
    assert info["iterations"] == len(R.rho_rel)


def test_ergodic_average_restarts_with_a_warm_start():
    P = synth.random_instance(21, horizon=6, max_children=3)
    steps = H.tiny_steps(P)
    R1 = _ergodic(P, steps, 50)
    nx = P["net"]["n_x"]
    y = H.stack_y(R1.y)
    R2 = _ergodic(P, steps, 30, y0=(y[:, :nx], y[:, nx:2 * nx], y[:, 2 * nx:]))
    g = H.Gpu(P, steps=steps)
    try:
        g.solve(50, ergodic=1)
        _check(g, R1, FP64_TOL)
        g.solve(30, warm=1, ergodic=1)
        _check(g, R2, FP64_TOL)
    finally:
        g.close()


def test_ergodic_average_in_graphs_equals_plain_launches():
    P = synth.random_instance(21, horizon=6, max_children=3)
    steps = H.tiny_steps(P)
    R = _ergodic(P, steps, 200)
    g = H.Gpu(P, steps=steps)
    try:
        for use_graph, ergodic in ((1, 1), (1, 0), (1, 1), (0, 1)):
            g.solve(200, ergodic=ergodic, use_graph=use_graph, check_every=64)
            if ergodic:
                _check(g, R, FP64_TOL)
    finally:
        g.close()


def test_forest_trees_average_up_to_their_own_stop():
    members = synth.forest_members(7, 5, max_horizon=7)
    F = synth.forest(members)
    n = len(F["tree"]["parent"])
    n_u = F["net"]["n_u"]
    steps = {"s": np.zeros(n), "z": np.zeros(n), "p": np.zeros((n, n_u))}
    per = []
    for r, P in enumerate(members):
        st = H.tiny_steps(P)
        idx = F["members"][r]
        for k in ("s", "z", "p"):
            steps[k][idx] = st[k]
        per.append(st)
    tol, cap = 2e-4, 4000
    g = H.Gpu(F, steps=steps, schedule=4)
    try:
        g.solve(cap, tol=tol, check_every=32, ergodic=1)
        ub, xb = g.bars()
    finally:
        g.close()
    counts = set()
    for r, P in enumerate(members):
        R = _ergodic(P, per[r], cap, tol=tol)
        counts.add(len(R.rho_rel))
        idx = F["members"][r]
        assert max(H.relerr(ub[idx], R.ubar), H.relerr(xb[idx], R.xbar)) <= FP64_TOL, r
    assert len(counts) > 1


def test_static_entry_refuses_the_ergodic_average():
    import paper_1604_01074_gb300 as smpc
    P = synth.tiny(0)
    g = H.Gpu(P, steps=H.tiny_steps(P))
    try:
        with pytest.raises(smpc.SmpcError) as ei:
            smpc.smpc_solve_static(g.fac, P["p"], P["q"], P["dhat"], P["alpha2"], eps=P["eps"], max_iters=10,
                                   ergodic=1)
        assert ei.value.code == smpc.SMPC_EINVAL
    finally:
        g.close()
