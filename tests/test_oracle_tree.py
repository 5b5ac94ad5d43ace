"""Pins for the node convention and variable layout: Table 1 of the paper.

Reading under test: one node per stage 0..N-1 holding (u_j, x_{j+1}); the root is
unique; each node contributes n_x + n_u primal and 2 n_x + n_u dual variables.
"""
import json
import os

import numpy as np

import synth
from oracle import Tree

HERE = os.path.dirname(__file__)


def test_table1_variable_counts():
    g = json.load(open(os.path.join(HERE, "golden", "table1.json")))
    n_x, n_u, N = g["n_x"], g["n_u"], g["horizon"]
    for row in g["rows"]:
        t = synth.make_tree(row["branching"], N, row["scenarios"])
        tree = Tree(t["parent"], t["prob"])
        assert len(tree.leaves) == row["scenarios"]
        assert tree.horizon == N
        primal = tree.n * (n_x + n_u)
        dual = tree.n * (2 * n_x + n_u)
        assert primal == row["primal"], row["name"]
        if row.get("dual_misprint"):
            assert dual == 32640 and row["dual"] == 32540
        else:
            assert dual == row["dual"], row["name"]


def test_tree_probabilities_consistent():
    # Sec. III-C: children's probabilities add up to the parent's; each stage sums to one
    for t in (synth.tiny()["tree"], synth.barcelona()["tree"], synth.random_instance(4)["tree"]):
        tree = Tree(t["parent"], t["prob"])
        for m in range(tree.n):
            if tree.children[m]:
                assert abs(sum(tree.prob[c] for c in tree.children[m]) - tree.prob[m]) < 1e-12
        for S in tree.nodes_at:
            assert abs(tree.prob[S].sum() - 1.0) < 1e-12


def test_workload_sizes():
    assert Tree(synth.tiny()["tree"]["parent"], synth.tiny()["tree"]["prob"]).n == 15
    b = synth.barcelona()["tree"]
    assert len(b["parent"]) == 2081
    assert int(np.sum(np.bincount(b["parent"][1:]) > 0)) == 2081 - 100
