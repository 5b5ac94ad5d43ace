"""The serving loop (smpc_server_*): solves of trees of different sizes and precisions
admitted into concurrent slots give the same results as each solved alone; admission
respects the device-memory budget; a controller's steps warm-start in order."""
import time

import numpy as np
import pytest

import synth
from tests import harness as H

pytestmark = pytest.mark.gpu


def _instances():
    return [
        ("tiny_f64", synth.tiny(0), 0),
        ("random_f32", synth.random_instance(31, horizon=8, max_children=3), 1),
        ("random_bf16", synth.random_instance(32, n_x=5, n_u=9, n_d=4, n_e=2, horizon=10, max_children=2), 2),
        ("wide_f32", synth.custom(33, 6, 10, 5, 2, synth.make_tree([6, 3], 6)), 1),
        ("chain_f64", synth.custom(34, 3, 5, 3, 1, synth.make_tree([1], 9)), 0),
    ]


def _wait(smpc, server, ticket, timeout=120.0, **out):
    t0 = time.time()
    while True:
        r = smpc.smpc_poll(server, ticket, **out)
        if r is not None:
            return r
        assert time.time() - t0 < timeout, "ticket did not complete"
        time.sleep(0.0005)


def _solve_alone(g, P, iters, tol, warm=0):
    u0 = np.zeros(g.n_u)
    info = g.smpc.smpc_solve(g.fac, P["p"], P["q"], P["dhat"], P["alpha2"], eps=P["eps"], max_iters=iters, tol=tol,
                             warm_start=warm, sync=1, u=g.u, x=g.x, y=g.y, u0_host=u0)
    return info, u0, [t.clone() for t in (g.u, g.x, g.y)]


def test_results_same_alone_and_in_the_mix():
    """Each served result equals the same factor's solve alone (bit for bit), and both
    match the FP64 oracle run for the same iteration count with the same steps:
    float64 factors to 1e-9 elementwise, reduced precisions by the residual tolerance
    (1e-4) and the elementwise bounds of the full-size reduced-precision tests."""
    import torch

    import paper_1604_01074_gb300 as smpc
    iters, tol = 1500, 1e-3
    steps = {name: H.full_size_steps(P, power_iters=60) for name, P, _ in _instances()}
    gs = [(name, P, H.Gpu(P, steps=steps[name], precision=prec)) for name, P, prec in _instances()]
    try:
        alone = {name: _solve_alone(g, P, iters, tol) for name, P, g in gs}
        budget = sum(smpc.smpc_factor_device_bytes(g.fac) for _, _, g in gs)
        server = smpc.smpc_server_create(budget, 3)
        try:
            tickets = []
            for rep in range(2):  # every instance twice, interleaved, all in flight together
                for name, P, g in (gs if rep == 0 else gs[::-1]):
                    t = smpc.smpc_submit(server, g.fac, P["p"], P["q"], P["dhat"], P["alpha2"], eps=P["eps"],
                                         max_iters=iters, tol=tol)
                    tickets.append((name, P, g, t))
            for name, P, g, t in tickets:
                u0 = np.zeros(g.n_u)
                outs = [torch.zeros_like(a) for a in (g.u, g.x, g.y)]
                r = _wait(smpc, server, t, u=outs[0], x=outs[1], y=outs[2], u0_host=u0)
                info, u0_ref, ref = alone[name]
                assert r["iterations"] == info["iterations"], name
                assert r["rho_rel"] == info["rho_rel"], name
                assert np.array_equal(u0, u0_ref), name
                for a, b in zip(outs, ref):
                    assert bool((a == b).all()), name
                _check_against_oracle(name, P, g, steps[name], r, outs)
        finally:
            smpc.smpc_server_destroy(server)
    finally:
        for _, _, g in gs:
            g.close()


def _check_against_oracle(name, P, g, steps, r, outs):
    prec = {n: p for n, _, p in _instances()}[name]
    R = H.oracle_run(P, steps, r["iterations"])
    u, x, y = (t.double().cpu().numpy() for t in outs)
    err = max(H.relerr(u, R.u), H.relerr(x, R.x), H.relerr(y, H.stack_y(R.y)))
    bound = {0: 1e-9, 1: 1e-4, 2: 2e-3}[prec]
    assert err <= bound, (name, err)
    assert abs(r["rho_rel"] - R.rho_rel[-1]) <= (1e-9 if prec == 0 else 1e-4), (name, r["rho_rel"], R.rho_rel[-1])
    if prec == 0:  # float64 stops at the oracle's first iterate with rho_rel <= tol
        assert R.rho_rel[-1] <= 1e-3 or r["iterations"] == 1500, name


def test_admission_by_device_memory():
    import paper_1604_01074_gb300 as smpc
    insts = _instances()[:3]
    gs = [(P, H.Gpu(P, precision=prec)) for _, P, prec in insts]
    try:
        sizes = [smpc.smpc_factor_device_bytes(g.fac) for _, g in gs]
        server = smpc.smpc_server_create(max(sizes), 3)  # room for one factor at a time
        try:
            big = H.Gpu(synth.barcelona(0), precision=1)
            try:
                with pytest.raises(smpc.SmpcError) as ei:
                    smpc.smpc_submit(server, big.fac, big.P["p"], big.P["q"], big.P["dhat"], big.P["alpha2"])
                assert ei.value.code == smpc.SMPC_EBUSY
            finally:
                big.close()
            ts = [smpc.smpc_submit(server, g.fac, P["p"], P["q"], P["dhat"], P["alpha2"], eps=P["eps"],
                                   max_iters=400) for P, g in gs]
            res = [_wait(smpc, server, t) for t in ts]
            assert all(r["iterations"] == 400 for r in res)
            with pytest.raises(smpc.SmpcError) as ei:
                smpc.smpc_poll(server, ts[0])  # released once returned as done
            assert ei.value.code == smpc.SMPC_EINVAL
        finally:
            smpc.smpc_server_destroy(server)
    finally:
        for _, g in gs:
            g.close()


def test_closed_loop_steps_warm_start_in_order():
    """Alg. 2 through the server: each step warm-starts from the previous step's duals,
    exactly as consecutive smpc_solve calls on a twin factor do."""
    import paper_1604_01074_gb300 as smpc
    P = synth.random_instance(35, horizon=6, max_children=3)
    # one pinned schedule for both: the autotuner could pick different (equally valid)
    # schedules for the two factors, whose float32 results differ in rounding
    twin, served = H.Gpu(P, precision=1, schedule=2), H.Gpu(P, precision=1, schedule=2)
    server = smpc.smpc_server_create(10 * smpc.smpc_factor_device_bytes(served.fac), 2)
    try:
        rng = np.random.default_rng(5)
        for k in range(3):
            p = P["p"] * (1 + 0.05 * rng.standard_normal(P["p"].shape))
            Pk = dict(P, p=p)
            info, u0_ref, _ = _solve_alone(twin, Pk, 300, 0.0, warm=int(k > 0))
            t = smpc.smpc_submit(server, served.fac, p, P["q"], P["dhat"], P["alpha2"], eps=P["eps"], max_iters=300,
                                 warm_start=int(k > 0))
            u0 = np.zeros(served.n_u)
            r = _wait(smpc, server, t, u0_host=u0)
            assert r["rho_rel"] == info["rho_rel"], k
            assert np.array_equal(u0, u0_ref), k
    finally:
        smpc.smpc_server_destroy(server)
        twin.close()
        served.close()


def test_admission_after_solves_that_grow_their_factors():
    """A solve with more iterations than any earlier one on its factor grows the factor's
    iteration buffers; admission must release exactly what it counted, so that later
    requests keep being admitted (a budget room for two factors, many rounds)."""
    import paper_1604_01074_gb300 as smpc
    insts = _instances()[:3]
    gs = [(P, H.Gpu(P, precision=prec)) for _, P, prec in insts]
    try:
        sizes = sorted(smpc.smpc_factor_device_bytes(g.fac) for _, g in gs)
        server = smpc.smpc_server_create(sizes[-1] + sizes[-2] + (1 << 20), 2)
        try:
            for rnd in range(4):
                iters = 1500 + 2000 * rnd  # every round beyond the factors' buffers so far
                ts = [smpc.smpc_submit(server, g.fac, P["p"], P["q"], P["dhat"], P["alpha2"], eps=P["eps"],
                                       max_iters=iters) for P, g in gs]
                res = [_wait(smpc, server, t, timeout=60.0) for t in ts]
                assert all(r["iterations"] == iters for r in res), rnd
        finally:
            smpc.smpc_server_destroy(server)
    finally:
        for _, g in gs:
            g.close()
