"""Oracle pin on the tree bookkeeping: the method does not depend on how the nodes of a
stage are numbered.

Algorithm 1 and the prox act node by node, through each node's parent, children, stage and
probability (Sec. III-C, Sec. IV-B); nothing in the iteration refers to the position of a
node within its stage.  Renumbering the nodes of every stage by a permutation (parents
still before their children) and carrying the per-node data along (forecast deviations,
probabilities, step sizes) must therefore give the same iterates, permuted, at every
iteration - not only at the solution.  A mistake that reads a node's data by position,
assumes a node's children are numbered together, or mixes node and stage indices fails
this on the ragged trees with random probabilities used here.
"""
import numpy as np
import pytest

import oracle
import synth


def _relabel(P, seed):
    """P with the nodes of every stage renumbered by a random permutation; new_of[m] is the
    new number of node m."""
    rng = np.random.default_rng(seed)
    par = np.asarray(P["tree"]["parent"])
    T = oracle.Tree(par, P["tree"]["prob"])
    order = np.concatenate([rng.permutation(T.nodes_at[j]) for j in range(T.horizon)])
    new_of = np.empty(T.n, dtype=np.int64)
    new_of[order] = np.arange(T.n)
    par2 = np.array([-1 if par[m] < 0 else new_of[par[m]] for m in order])
    tree2 = dict(P["tree"], parent=par2, prob=np.asarray(P["tree"]["prob"])[order],
                 stage=np.asarray(P["tree"]["stage"])[order])
    return dict(P, tree=tree2, eps=P["eps"][order]), new_of


def _run(P, iters, steps=None):
    T = oracle.Tree(P["tree"]["parent"], P["tree"]["prob"])
    fac = oracle.factor(P["net"], P["cost"])
    cu = oracle.cost_update(fac, P["cost"], T, P["alpha2"], P["dhat"], P["eps"], P["q"])
    st = oracle.jacobi_steps(fac, T) if steps is None else steps
    return oracle.apg(fac, T, cu, P["cost"], P["p"], st, iters), st


@pytest.mark.parametrize("P", [synth.random_instance(21, horizon=6, max_children=3),
                               synth.random_instance(22, n_x=4, n_u=7, n_d=4, n_e=2, horizon=5, max_children=4),
                               synth.tiny(0)], ids=["random_a", "random_b", "tiny"])
def test_renumbering_the_nodes_of_a_stage_permutes_the_iterates(P):
    iters = 200
    R, st = _run(P, iters)
    P2, new_of = _relabel(P, 7)
    st2 = {"s": st["s"][np.argsort(new_of)], "z": st["z"][np.argsort(new_of)], "p": st["p"][np.argsort(new_of)]}
    R2, _ = _run(P2, iters, st2)
    scale = lambda a: 1.0 + np.abs(a).max()  # noqa: E731
    for a, b in ((R.u, R2.u), (R.x, R2.x), (R.y[0], R2.y[0]), (R.y[1], R2.y[1]), (R.y[2], R2.y[2])):
        assert np.abs(b[new_of] - a).max() <= 1e-10 * scale(a)
    np.testing.assert_allclose(R2.rho_rel, R.rho_rel, rtol=1e-9, atol=0)
    # the steps of the renumbered tree, computed on it, are the same steps renumbered
    _, st_own = _run(P2, 1)
    for k in ("s", "z", "p"):
        np.testing.assert_allclose(st_own[k][new_of], st[k], rtol=1e-12, atol=0)


def test_renumbering_pin_catches_node_data_read_by_position():
    """Planted: the renumbered tree keeps the forecast deviations in the old order (a node's
    data read by its position): the iterates no longer match."""
    P = synth.random_instance(21, horizon=6, max_children=3)
    R, st = _run(P, 200)
    P2, new_of = _relabel(P, 7)
    P2 = dict(P2, eps=P["eps"])
    st2 = {k: st[k][np.argsort(new_of)] for k in ("s", "z", "p")}
    R2, _ = _run(P2, 200, st2)
    assert np.abs(R2.u[new_of] - R.u).max() > 1e-3 * (1.0 + np.abs(R.u).max())
