"""Seeded scenario-tree builders (input data only; none of the solver's arithmetic).

A tree is described the way the solver consumes it (Sec. III-C of the paper):
nodes are numbered in breadth-first order grouped by stage, ``parent[0] == -1``
marks the root, every other node's parent is at the previous stage, and leaves
all sit at stage ``horizon - 1``.  Scenarios are the root-to-leaf paths; with
equiprobable scenarios a node's probability is (leaves below it) / (number of
leaves), which makes the probabilities of the children of a node add up to the
probability of the node (Sec. III-C).

Branching factors follow Table 1's convention: ``branching[j]`` is the maximum
number of children of a node at stage ``j``; stages past the list have one
child per node.  When the requested number of scenarios is smaller than the
product of the factors, the last branching stage gets a near-even fan-out
(no node above its maximum) that reaches exactly that many leaves.
"""
from __future__ import annotations

import numpy as np


def _stage_counts(branching, horizon, n_scenarios):
    """Number of children of each node at every stage, stage by stage."""
    branching = [int(b) for b in branching]
    nb = 0
    for j, b in enumerate(branching):
        if b > 1 and j < horizon - 1:
            nb = j + 1
    full = 1
    for b in branching[:nb]:
        full *= b
    if n_scenarios is None:
        n_scenarios = full
    if nb == 0:
        if n_scenarios != 1:
            raise ValueError("a tree without branching has exactly one scenario")
    prev = full // branching[nb - 1] if nb else 1
    if nb and not (prev <= n_scenarios <= full):
        raise ValueError(f"{n_scenarios} scenarios cannot be reached with branching {branching[:nb]}")
    fanouts = []  # fanouts[j] = list of child counts for the nodes of stage j
    width = 1
    for j in range(horizon - 1):
        if j < nb - 1:
            fan = [branching[j]] * width
        elif j == nb - 1:
            base, extra = divmod(n_scenarios, width)
            fan = [base + (1 if i < extra else 0) for i in range(width)]
            if max(fan) > branching[j] or min(fan) < 1:
                raise ValueError("near-even fan-out exceeds the maximum branching factor")
        else:
            fan = [1] * width
        fanouts.append(fan)
        width = sum(fan)
    return fanouts


def tree_from_fanouts(fanouts):
    """parent[] (BFS order by stage) from per-stage lists of child counts."""
    parent = [-1]
    first_of_stage = 0
    width = 1
    for fan in fanouts:
        assert len(fan) == width
        for i, c in enumerate(fan):
            parent.extend([first_of_stage + i] * c)
        first_of_stage += width
        width = sum(fan)
    return np.asarray(parent, dtype=np.int32)


def stages_of(parent):
    parent = np.asarray(parent)
    stage = np.zeros(len(parent), dtype=np.int32)
    for n in range(1, len(parent)):
        stage[n] = stage[parent[n]] + 1
    return stage


def uniform_scenario_probabilities(parent):
    """p_n = (leaves under n) / (number of leaves): equiprobable scenarios."""
    parent = np.asarray(parent)
    n = len(parent)
    has_child = np.zeros(n, dtype=bool)
    has_child[parent[1:]] = True
    leaves = np.where(~has_child, 1.0, 0.0)
    for m in range(n - 1, 0, -1):  # BFS order: children after parents
        leaves[parent[m]] += leaves[m]
    return leaves / leaves[0]


def make_tree(branching, horizon, n_scenarios=None):
    """Scenario tree with Table 1's branching convention and equiprobable scenarios."""
    fanouts = _stage_counts(branching, horizon, n_scenarios)
    parent = tree_from_fanouts(fanouts)
    return {"parent": parent, "stage": stages_of(parent),
            "prob": uniform_scenario_probabilities(parent), "horizon": int(horizon)}


def random_tree(rng, horizon, max_children=3, branch_stages=None, p_branch=0.5):
    """Irregular tree for edge cases: branching at arbitrary stages, uneven fan-out,
    non-uniform (random) scenario probabilities."""
    if branch_stages is None:
        branch_stages = [j for j in range(horizon - 1) if rng.random() < p_branch]
    fanouts = []
    width = 1
    for j in range(horizon - 1):
        if j in branch_stages:
            fan = [int(rng.integers(1, max_children + 1)) for _ in range(width)]
        else:
            fan = [1] * width
        fanouts.append(fan)
        width = sum(fan)
    parent = tree_from_fanouts(fanouts)
    n = len(parent)
    # random conditional probabilities: each node splits its mass among its children
    w = rng.uniform(0.2, 1.0, size=n)
    prob = np.zeros(n)
    prob[0] = 1.0
    child_sum = np.zeros(n)
    for m in range(1, n):
        child_sum[parent[m]] += w[m]
    for m in range(1, n):
        prob[m] = prob[parent[m]] * w[m] / child_sum[parent[m]]
    return {"parent": parent, "stage": stages_of(parent), "prob": prob, "horizon": int(horizon)}


def tree_from_fanouts_dict(fanouts):
    """Tree dict (equiprobable scenarios) from explicit per-stage child counts."""
    parent = tree_from_fanouts(fanouts)
    return {"parent": parent, "stage": stages_of(parent), "prob": uniform_scenario_probabilities(parent),
            "horizon": len(fanouts) + 1}
