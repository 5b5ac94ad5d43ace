"""One tree split over two ranks (CPU, gloo): the host loop of the sharded solve
(paper_1604_01074_gb300.shard.sharded_solve, the same code the GPUs run) with a CPU
stand-in for each rank's phases (tests/shard_cpu.py).  The union of the ranks' rows
equals the FP64 oracle's APG iterates on the whole tree, for fixed iteration counts and
for a tolerance stop, with the chains of one cut parent split across the ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _case(name):
    import synth
    from tests import harness as H
    if name == "barcelona_small":
        P = synth.barcelona(0, branching=(2, 2), n_scenarios=4)  # 4 chains of 22 nodes under 2 cut parents
        return P, H.full_size_steps(P)
    P = synth.random_instance(21, horizon=6, max_children=3)
    import oracle
    tree, fac, _ = H.oracle_build(P)
    return P, oracle.jacobi_steps(fac, tree)


def _worker(rank, world, port, name, split, iters, tol, out):
    import torch.distributed as dist

    from paper_1604_01074_gb300.shard import sharded_solve
    from tests.shard_cpu import CpuShard, chains_of
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    P, steps = _case(name)
    n_chains = len(chains_of(P["tree"]["parent"])[0])
    bounds = [0, split, n_chains]
    sh = CpuShard(P, steps, bounds[rank], bounds[rank + 1])
    step = {k: P[k] for k in ("p", "q", "dhat", "alpha2", "eps")}
    info = sharded_solve(sh, step, max_iters=iters, tol=tol, check_every=8)
    S = np.asarray(sh.nodes)
    out[rank] = (S, sh.x[S], sh.u[S], sh.y[0][S], info)
    dist.barrier()
    dist.destroy_process_group()


def _run(name, split, iters, tol):
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, name, split, iters, tol, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
            assert p.exitcode == 0
        return dict(out)


@pytest.mark.parametrize("name,split", [("barcelona_small", 1), ("barcelona_small", 3), ("random", 2)])
def test_two_ranks_match_the_oracle(name, split):
    from tests import harness as H
    res = _run(name, split, 40, 0.0)
    P, steps = _case(name)
    R = H.oracle_run(P, steps, 40)
    Y = H.stack_y(R.y)
    seen = np.zeros(len(P["tree"]["parent"]), bool)
    for rank, (S, x, u, y, info) in res.items():
        assert info["iterations"] == 40
        assert abs(info["rho"] - R.rho[-1]) <= 1e-9 * (1 + R.rho[-1])
        for a, b in ((x, R.x[S]), (u, R.u[S]), (y, Y[S])):
            assert np.abs(a - b).max() <= 1e-9 * (1 + np.abs(b).max()), rank
        seen[S] = True
    assert seen.all()  # every node is some rank's (the top on both)


def test_two_ranks_stop_together_at_the_oracle_iterate():
    import oracle
    from tests import harness as H
    tol = 2e-3
    res = _run("random", 2, 3000, tol)
    P, steps = _case("random")
    tree, fac, cu = H.oracle_build(P)
    R = oracle.apg(fac, tree, cu, P["cost"], P["p"], steps, 3000, tol=tol)
    k = len(R.rho_rel)
    Y = H.stack_y(R.y)
    for rank, (S, x, u, y, info) in res.items():
        assert info["iterations"] == k, (rank, info, k)
        for a, b in ((x, R.x[S]), (u, R.u[S]), (y, Y[S])):
            assert np.abs(a - b).max() <= 1e-9 * (1 + np.abs(b).max()), rank
