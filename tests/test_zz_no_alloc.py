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


def _compare_static_to_solve(P, steps, iters, tol=0.0):
    g = H.Gpu(P, steps=steps)
    try:
        ref = g.solve(iters, tol=tol)
        ref_u, ref_x, ref_y = g.arrays()
        for call in range(2):  # two calls in a row share (and reuse) the static scratch
            u, x, y = _outputs(g)
            hist = np.zeros((iters, 3))
            u0 = np.zeros(g.n_u)
            info = g.smpc.smpc_solve_static(g.fac, P["p"], P["q"], P["dhat"], P["alpha2"], eps=P["eps"],
                                            max_iters=iters, tol=tol, sync=1, u=u, x=x, y=y, u0_host=u0,
                                            history_host=hist)
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
