"""A general state matrix A (App. B) through the C ABI against the FP64 oracle, element by
element: s_n = xi_n + A' sum of the children's s in the backward sweep and
x_n = A x_parent + Bbar v_n + e_n in the forward sweep, on the node-parallel schedule (2),
which is the one that carries A.  Bars: float64 1e-9, float32 1e-4 (relative to 1 + the
largest entry), as in the A = I parity tests."""
import numpy as np
import pytest

import oracle
import synth
from tests import harness as H

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-9
FP32_TOL = 1e-4


def _instances():
    return {
        "tiny": synth.general_dynamics(synth.tiny(0)),
        "random_a": synth.general_dynamics(H.edge_instances()["random_a"], 1),
        "late_branch": synth.general_dynamics(H.edge_instances()["late_branch"], 2),
        "chain": synth.general_dynamics(H.edge_instances()["chain"], 3),
        "root_fan": synth.general_dynamics(H.edge_instances()["root_fan"], 4),
    }


def _compare(P, iters, precision=0, shared=0, bound=FP64_TOL):
    steps = H.tiny_steps(P)
    R = H.oracle_run(P, steps, iters)
    g = H.Gpu(P, steps=steps, schedule=0, precision=precision, shared_packs=shared)
    try:
        assert g.smpc.smpc_factor_schedule(g.fac)[0] == 2  # the schedule that carries A
        info = g.solve(iters)
        u, x, y = g.arrays()
    finally:
        g.close()
    assert info["iterations"] == iters
    e = (H.relerr(u, R.u), H.relerr(x, R.x), H.relerr(y, H.stack_y(R.y)))
    assert max(e) <= bound, e
    return info, R


@pytest.mark.parametrize("name", list(_instances()))
@pytest.mark.parametrize("iters", [1, 10, 200])
def test_general_A_fp64(name, iters):
    P = _instances()[name]
    info, R = _compare(P, iters)
    np.testing.assert_allclose(info["history"][:, 0], R.rho, rtol=1e-7, atol=1e-9)


@pytest.mark.parametrize("shared", [0, 1])
def test_general_A_fp64_shared_packs(shared):
    _compare(_instances()["random_a"], 100, shared=shared)


@pytest.mark.parametrize("shared", [0, 1])
def test_general_A_fp32(shared):
    _compare(_instances()["random_a"], 100, precision=1, shared=shared, bound=FP32_TOL)


def test_general_A_full_size():
    """The 2081-node Barcelona-shaped tree with leaking, exchanging tanks: float64 and float32
    against the oracle after 20 iterations."""
    P = synth.general_dynamics(synth.barcelona(0))
    steps = H.full_size_steps(P)
    iters = 20
    R = H.oracle_run(P, steps, iters)
    for prec, bound in ((0, FP64_TOL), (1, FP32_TOL)):
        g = H.Gpu(P, steps=steps, precision=prec)
        try:
            g.solve(iters)
            u, x, y = g.arrays()
        finally:
            g.close()
        e = (H.relerr(u, R.u), H.relerr(x, R.x), H.relerr(y, H.stack_y(R.y)))
        assert max(e) <= bound, (prec, e)


def test_general_A_tolerance_stop_matches_oracle():
    P = _instances()["tiny"]
    steps = H.tiny_steps(P)
    tree, fac, cu = H.oracle_build(P)
    tol, cap = 1e-4, 20000
    R = oracle.apg(fac, tree, cu, P["cost"], P["p"], steps, cap, tol=tol)
    g = H.Gpu(P, steps=steps)
    try:
        info = g.solve(cap, tol=tol, check_every=32)
        u, x, y = g.arrays()
    finally:
        g.close()
    assert info["iterations"] == len(R.rho_rel)
    assert max(H.relerr(u, R.u), H.relerr(x, R.x)) <= FP64_TOL


def test_general_A_lambda_is_the_dense_eigenvalue():
    """Without preconditioning, lambda = 1 / largest eigenvalue of the dual Hessian, which the
    oracle forms densely (column by column from Algorithm 1 with A)."""
    P = _instances()["tiny"]
    tree, fac, _ = H.oracle_build(P)
    L = oracle.lipschitz_dense(oracle.dense_dual_hessian(fac, tree))
    g = H.Gpu(P, precondition=0, power_iters=600, lambda_margin=1e-12)
    try:
        lam = g.smpc.smpc_factor_steps(g.fac, g.n, g.n_u)[0]
    finally:
        g.close()
    assert abs(1.0 / lam - L) <= 1e-6 * L


@pytest.mark.parametrize("schedule", [1, 3, 4])
def test_general_A_refused_on_the_chain_schedules(schedule):
    import paper_1604_01074_gb300 as smpc
    P = _instances()["tiny"]
    tree = smpc.smpc_tree_create(P["tree"]["parent"], P["tree"]["prob"])
    try:
        with pytest.raises(smpc.SmpcError) as ei:
            smpc.smpc_factor(tree, P["net"], P["cost"], precision=0, lam=1e-3, schedule=schedule)
        assert ei.value.code == smpc.SMPC_ENOTSUP
    finally:
        smpc.smpc_tree_destroy(tree)


def test_general_A_static_entry_and_shard_refusal():
    import paper_1604_01074_gb300 as smpc
    P = _instances()["random_a"]
    steps = H.tiny_steps(P)
    R = H.oracle_run(P, steps, 50)
    g = H.Gpu(P, steps=steps)
    try:
        smpc.smpc_solve_static(g.fac, P["p"], P["q"], P["dhat"], P["alpha2"], eps=P["eps"], max_iters=50,
                               u=g.u, x=g.x, y=g.y)
        u, x, _ = g.arrays()
        assert max(H.relerr(u, R.u), H.relerr(x, R.x)) <= FP64_TOL
        with pytest.raises(smpc.SmpcError) as ei:
            smpc.smpc_shard_create(g.fac, 0, 1)
        assert ei.value.code == smpc.SMPC_ENOTSUP
    finally:
        g.close()
