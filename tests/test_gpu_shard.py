"""The sharded solve through the C ABI (smpc_shard_*): one tree's chains split over two
ranks, each running the library's kernels on its own shard, the exchange between them
done by the host loop of paper_1604_01074_gb300.shard over gloo (through host memory).
Both ranks run on the one GPU of this machine as separate processes: their kernels never
wait on each other (every exchange goes through the host between launches).  The
union of the ranks' rows equals the FP64 oracle's APG iterates on the whole tree."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _case(name):
    import oracle
    import synth
    from tests import harness as H
    if name == "barcelona_small":
        P = synth.barcelona(0, branching=(2, 2), n_scenarios=4)
        return P, H.full_size_steps(P)
    if name == "barcelona":
        P = synth.barcelona(0)
        return P, H.full_size_steps(P)
    P = synth.random_instance(21, horizon=6, max_children=3)
    tree, fac, _ = H.oracle_build(P)
    return P, oracle.jacobi_steps(fac, tree)


def _worker(rank, world, port, name, prec, split, iters, tol, out):
    import torch
    import torch.distributed as dist

    import paper_1604_01074_gb300 as smpc
    from paper_1604_01074_gb300.shard import LibraryShard, sharded_solve
    torch.cuda.set_device(0)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    P, steps = _case(name)
    t, net = P["tree"], P["net"]
    n = len(t["parent"])
    tree = smpc.smpc_tree_create(t["parent"], t["prob"])
    n_chains = smpc.smpc_tree_info_get(tree)["n_chains"]
    fac = smpc.smpc_factor(tree, net, P["cost"], precision=prec, steps=steps)
    bounds = [0, split if split > 0 else n_chains // 2, n_chains]
    sh = LibraryShard(fac, prec, bounds[rank], bounds[rank + 1], n, net["n_x"], net["n_u"])
    step = {k: P[k] for k in ("p", "q", "dhat", "alpha2", "eps")}
    info = sharded_solve(sh, step, max_iters=iters, tol=tol, check_every=16)
    S = np.asarray(sh.nodes, dtype=np.int64)
    out[rank] = (S, sh.x.double().cpu().numpy()[S], sh.u.double().cpu().numpy()[S], sh.y.double().cpu().numpy()[S],
                 info)
    sh.close()
    smpc.smpc_factor_destroy(fac)
    smpc.smpc_tree_destroy(tree)
    dist.barrier()
    dist.destroy_process_group()


def _run(name, prec, split, iters, tol):
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, name, prec, split, iters, tol, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(600)
            assert p.exitcode == 0
        return dict(out)


@pytest.mark.parametrize("name,prec,split,iters,bound", [
    ("barcelona_small", 0, 1, 40, 1e-9),   # the chains of one cut parent on both ranks
    ("random", 0, 2, 60, 1e-9),            # a ragged tree
    ("barcelona", 0, 37, 20, 1e-9),        # 2081 nodes, 100 chains split 37 / 63
    ("barcelona", 1, 0, 20, 1e-4),         # float32 packs, the float32 bar of the parity tests
])
def test_two_ranks_match_the_oracle(name, prec, split, iters, bound):
    from tests import harness as H
    res = _run(name, prec, split, iters, 0.0)
    P, steps = _case(name)
    R = H.oracle_run(P, steps, iters)
    Y = H.stack_y(R.y)
    seen = np.zeros(len(P["tree"]["parent"]), bool)
    for rank, (S, x, u, y, info) in res.items():
        assert info["iterations"] == iters
        for a, b in ((x, R.x), (u, R.u), (y, Y)):
            assert np.abs(a - b[S]).max() <= bound * (1 + np.abs(b).max()), rank
        assert abs(info["rho_rel"] - R.rho_rel[-1]) <= (1e-9 if prec == 0 else 1e-4)
        seen[S] = True
    assert seen.all()


def test_two_ranks_stop_together_at_the_oracle_iterate():
    import oracle
    from tests import harness as H
    tol = 2e-3
    res = _run("random", 0, 2, 3000, tol)
    P, steps = _case("random")
    tree, fac, cu = H.oracle_build(P)
    R = oracle.apg(fac, tree, cu, P["cost"], P["p"], steps, 3000, tol=tol)
    k = len(R.rho_rel)
    Y = H.stack_y(R.y)
    for rank, (S, x, u, y, info) in res.items():
        assert info["iterations"] == k, (rank, info, k)
        for a, b in ((x, R.x), (u, R.u), (y, Y)):
            assert np.abs(a - b[S]).max() <= 1e-9 * (1 + np.abs(b).max()), rank
