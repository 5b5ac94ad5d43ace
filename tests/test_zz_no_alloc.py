"""smpc_solve_static, the solve entry point that allocates no memory (its scratch lives
in the library's static device array), against smpc_solve on the same factor.

Callers that cannot allocate while they run - a controller that must return its move
within every sampling period, a service with a fixed device-memory budget - use it
instead of smpc_solve.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import harness as H

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-9


def _outputs(g):
    import torch
    return torch.zeros_like(g.u), torch.zeros_like(g.x), torch.zeros_like(g.y)


def _compare_static_to_solve(P, steps, iters, tol=0.0, precision=0, polish_iters=0, before_each=None):
    """smpc_solve once, then smpc_solve_static twice in a row on the same factor; both
    static calls must give smpc_solve's results.  before_each() runs before each static
    call (e.g. another factor's static solve, which leaves foreign data in the array)."""
    g = H.Gpu(P, steps=steps, precision=precision)
    try:
        u0r = np.zeros(g.n_u)
        histr = np.zeros((iters, 3))
        ref = g.smpc.smpc_solve(g.fac, P["p"], P["q"], P["dhat"], P["alpha2"], eps=P["eps"], max_iters=iters, tol=tol,
                                sync=1, u=g.u, x=g.x, y=g.y, u0_host=u0r, history_host=histr,
                                polish_iters=polish_iters)
        ref["u0"] = u0r
        ref["history"] = histr[:max(ref["iterations"], 0)]
        ref_u, ref_x, ref_y = g.arrays()
        for call in range(2):  # two calls in a row share (and reuse) the static scratch
            if before_each is not None:
                before_each()
            u, x, y = _outputs(g)
            hist = np.zeros((iters, 3))
            u0 = np.zeros(g.n_u)
            info = g.smpc.smpc_solve_static(g.fac, P["p"], P["q"], P["dhat"], P["alpha2"], eps=P["eps"],
                                            max_iters=iters, tol=tol, sync=1, u=u, x=x, y=y, u0_host=u0,
                                            history_host=hist, polish_iters=polish_iters)
            assert info["iterations"] == ref["iterations"], call
            for got, want in ((u, ref_u), (x, ref_x), (y, ref_y)):
                assert H.relerr(got.double().cpu().numpy(), want) <= FP64_TOL, call
            assert abs(info["rho_rel"] - ref["rho_rel"]) <= FP64_TOL
            np.testing.assert_allclose(u0, ref["u0"], rtol=0, atol=FP64_TOL * (1 + np.abs(ref["u0"]).max()))
            it = info["iterations"]
            np.testing.assert_allclose(hist[:it], ref["history"], rtol=1e-9, atol=1e-12)
    finally:
        g.close()


def test_static_solve_matches_solve_ragged_tree():
    P = synth.random_instance(21, horizon=6, max_children=3)
    tree, fac, _ = H.oracle_build(P)
    _compare_static_to_solve(P, oracle.jacobi_steps(fac, tree), 120)


def test_static_solve_matches_solve_tolerance_stop():
    P = synth.tiny(0)
    _compare_static_to_solve(P, H.tiny_steps(P), 3000, tol=1e-3)


def test_static_solve_matches_solve_full_tree():
    P = synth.barcelona(0)
    tree, fac, _ = H.oracle_build(P)
    unit = H.closed_form_steps(fac, tree, 1.0)
    steps = H.closed_form_steps(fac, tree, 1.0 / (1.02 * H.oracle_power_lambda(fac, tree, unit, iters=30)))
    _compare_static_to_solve(P, steps, 40)


def test_static_solve_refuses_requests_beyond_its_scratch():
    import paper_1604_01074_gb300 as smpc
    P = synth.barcelona(0)
    tree, fac, _ = H.oracle_build(P)
    g = H.Gpu(P, steps=H.closed_form_steps(fac, tree, 1e-6))
    try:
        with pytest.raises(smpc.SmpcError) as ei:
            smpc.smpc_solve_static(g.fac, P["p"], P["q"], P["dhat"], P["alpha2"], eps=P["eps"], max_iters=2_000_000)
        assert ei.value.code == smpc.SMPC_EINVAL
        assert "static scratch" in str(ei.value)
    finally:
        g.close()


@pytest.mark.parametrize("precision,polish", [(1, 0), (2, 40)])
def test_static_solve_matches_solve_reduced_precision(precision, polish):
    """float32 packs, and bfloat16 packs with float32 anchors and a float32 polish (the
    anchored solve reads the factor's own anchor buffers)."""
    P = synth.random_instance(24, horizon=7, max_children=3)
    tree, fac, _ = H.oracle_build(P)
    _compare_static_to_solve(P, oracle.jacobi_steps(fac, tree), 150, precision=precision, polish_iters=polish)


def test_static_solve_does_not_depend_on_what_another_factor_left():
    """Before each compared call, a static solve of a larger, differently shaped factor
    (the 2081-node tree, float64) fills the shared array with its own data."""
    big_P = synth.barcelona(0)
    tree, fac, _ = H.oracle_build(big_P)
    big = H.Gpu(big_P, steps=H.closed_form_steps(fac, tree, 1e-6))
    try:
        def foreign():
            big.smpc.smpc_solve_static(big.fac, big_P["p"], big_P["q"], big_P["dhat"], big_P["alpha2"],
                                       eps=big_P["eps"], max_iters=30, sync=1)
        P = synth.random_instance(25, horizon=6, max_children=4)
        t2, f2, _ = H.oracle_build(P)
        _compare_static_to_solve(P, oracle.jacobi_steps(f2, t2), 90, precision=1, before_each=foreign)
    finally:
        big.close()


def test_solve_info_refuses_after_async_static_solve():
    """The host outputs of smpc_solve_static come with sync = 1; smpc_solve_info, which
    completes smpc_solve, refuses a factor whose last solve was static."""
    import torch
    P = synth.tiny(0)
    g = H.Gpu(P, steps=H.tiny_steps(P))
    try:
        g.smpc.smpc_solve_static(g.fac, P["p"], P["q"], P["dhat"], P["alpha2"], eps=P["eps"], max_iters=50, sync=0)
        torch.cuda.synchronize()
        with pytest.raises(g.smpc.SmpcError) as ei:
            g.smpc.smpc_solve_info(g.fac)
        assert ei.value.code == g.smpc.SMPC_EINVAL
        g.solve(20)  # smpc_solve completes through smpc_solve_info again
    finally:
        g.close()
