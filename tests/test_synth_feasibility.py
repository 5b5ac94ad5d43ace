"""The synthetic workloads keep the problem feasible (the paper does not state it; the
generator guarantees it): E has full row rank, and at every node some input inside the
box [u_min, u_max] satisfies the coupling E u + E_d d_n = 0 with that node's demand.
Checked by a feasibility linear program per node (scipy), not by the generator's own
construction."""
import numpy as np
import pytest

import synth


def _demands(P):
    return P["dhat"][P["tree"]["stage"]] + P["eps"]


def _box_feasible(E, Ed, d, lo, hi):
    from scipy.optimize import linprog
    res = linprog(np.zeros(E.shape[1]), A_eq=E, b_eq=-Ed @ d, bounds=list(zip(lo, hi)), method="highs")
    return res.status == 0


@pytest.mark.parametrize("mk,sample", [(lambda: synth.tiny(0), None), (lambda: synth.random_instance(3), None),
                                       (lambda: synth.barcelona(0), 60)])
def test_coupling_feasible_at_every_node(mk, sample):
    pytest.importorskip("scipy")
    P = mk()
    net, cost = P["net"], P["cost"]
    E, Ed = net["E"], net["Ed"]
    assert np.linalg.matrix_rank(E) == E.shape[0]
    d = _demands(P)
    nodes = np.arange(len(d))
    if sample is not None:  # a seeded sample of the nodes of the large tree
        nodes = np.random.default_rng(0).choice(nodes, size=sample, replace=False)
    for m in nodes:
        assert _box_feasible(E, Ed, d[m], cost["u_min"], cost["u_max"]), m


def test_batched_instances_feasible():
    """One instance on each of the four networks of the batched workload, 20 nodes each."""
    pytest.importorskip("scipy")
    rng = np.random.default_rng(1)
    for P in synth.batch_instances(0, count=4):
        E, Ed = P["net"]["E"], P["net"]["Ed"]
        assert np.linalg.matrix_rank(E) == E.shape[0]
        d = _demands(P)
        for m in rng.choice(len(d), size=20, replace=False):
            assert _box_feasible(E, Ed, d[m], P["cost"]["u_min"], P["cost"]["u_max"]), (P["name"], m)
