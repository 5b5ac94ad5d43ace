"""Batched solves (smpc_batch_*): factors on different networks - a forest of uneven
trees, single trees, mixed precisions - solved together, one launch per chunk of
iterations for the whole batch (a CUDA graph with one branch per factor, or the same
kernels on one stream per factor).  Each factor's result is bit for bit its result
solved alone, every forest tree stops on its own, and the float64 members match the
FP64 oracle run on each tree alone."""
import numpy as np
import pytest

import oracle
import synth
from tests import harness as H

pytestmark = pytest.mark.gpu


def _members():
    forest_members = synth.forest_members(7, 5, max_horizon=7)
    F = synth.forest(forest_members)
    n = len(F["tree"]["parent"])
    steps = {"s": np.zeros(n), "z": np.zeros(n), "p": np.zeros((n, F["net"]["n_u"]))}
    per = []
    for r, P in enumerate(forest_members):
        tree, fac, _ = H.oracle_build(P)
        st = oracle.jacobi_steps(fac, tree)
        for k in ("s", "z", "p"):
            steps[k][F["members"][r]] = st[k]
        per.append(st)
    tiny = synth.tiny(0)
    rnd = synth.random_instance(22, n_x=4, n_u=7, n_d=4, n_e=2, horizon=5, max_children=4)
    t2, f2, _ = H.oracle_build(rnd)
    cases = [("forest_f64", F, steps, 0), ("tiny_f64", tiny, H.tiny_steps(tiny), 0),
             ("random_f32", rnd, oracle.jacobi_steps(f2, t2), 1), ("forest_bf16", F, steps, 2)]
    return cases, forest_members, per


def _alone(g, P, iters, tol):
    u0 = np.zeros(len(P["q"]))
    info = g.smpc.smpc_solve(g.fac, P["p"], P["q"], P["dhat"], P["alpha2"], eps=P["eps"], max_iters=iters, tol=tol,
                             check_every=32, sync=1, u=g.u, x=g.x, y=g.y, u0_host=u0)
    return info, u0, [t.clone() for t in (g.u, g.x, g.y)]


@pytest.mark.parametrize("use_graph", [0, 1])
def test_batch_matches_each_factor_alone_and_the_oracle(use_graph):
    import torch

    import paper_1604_01074_gb300 as smpc
    cases, forest_members, per = _members()
    iters, tol = 3000, 2e-4
    gs = [(name, P, H.Gpu(P, steps=st, precision=prec, schedule=2)) for name, P, st, prec in cases]
    try:
        alone = {name: _alone(g, P, iters, tol) for name, P, g in gs}
        batch = smpc.smpc_batch_create([g.fac for _, _, g in gs])
        try:
            for rep in range(2):  # capture, then replay
                outs = [tuple(torch.zeros_like(t) for t in (g.u, g.x, g.y)) for _, _, g in gs]
                u0s = [np.zeros(len(P["q"])) for _, P, _ in gs]
                res = smpc.smpc_batch_solve(batch, [P for _, P, _ in gs], max_iters=iters, tol=tol, check_every=32,
                                            outputs=outs, u0_host=u0s, use_graph=use_graph)
                for (name, P, g), r, o, u0 in zip(gs, res, outs, u0s):
                    info, u0_ref, ref = alone[name]
                    assert r["iterations"] == info["iterations"], (name, rep)
                    assert r["rho_rel"] == info["rho_rel"], (name, rep)
                    assert np.array_equal(u0, u0_ref), (name, rep)
                    for a, b in zip(o, ref):
                        assert bool(torch.equal(a, b)), (name, rep)
            # the forest's trees, each against the oracle on that tree alone (float64)
            F = cases[0][1]
            g = gs[0][2]
            its, rr = smpc.smpc_solve_trees(g.fac, len(forest_members))
            u, x, y = (t.double().cpu().numpy() for t in outs[0])
            for r, P in enumerate(forest_members):
                tree, fac, cu = H.oracle_build(P)
                R = oracle.apg(fac, tree, cu, P["cost"], P["p"], per[r], iters, tol=tol)
                assert its[r] == len(R.rho_rel), r
                idx = F["members"][r]
                e = (H.relerr(u[idx], R.u), H.relerr(x[idx], R.x), H.relerr(y[idx], H.stack_y(R.y)))
                assert max(e) <= 1e-9, (r, e)
            # the tiny single tree against the oracle
            Pt, st = cases[1][1], cases[1][2]
            tree, fac, cu = H.oracle_build(Pt)
            R = oracle.apg(fac, tree, cu, Pt["cost"], Pt["p"], st, iters, tol=tol)
            u, x, y = (t.double().cpu().numpy() for t in outs[1])
            assert res[1]["iterations"] == len(R.rho_rel)
            assert max(H.relerr(u, R.u), H.relerr(x, R.x), H.relerr(y, H.stack_y(R.y))) <= 1e-9
        finally:
            smpc.smpc_batch_destroy(batch)
    finally:
        for _, _, g in gs:
            g.close()


def test_batch_refuses_a_repeated_factor():
    import paper_1604_01074_gb300 as smpc
    P = synth.tiny(0)
    g = H.Gpu(P, steps=H.tiny_steps(P))
    try:
        with pytest.raises(smpc.SmpcError) as ei:
            smpc.smpc_batch_create([g.fac, g.fac])
        assert ei.value.code == smpc.SMPC_EINVAL
    finally:
        g.close()
