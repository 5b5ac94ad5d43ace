"""Scenario-tree bookkeeping (Sec. III-C).

Nodes are given by a parent array in breadth-first order by stage; node n at
stage j holds the input u_j, the demand d_j and the state x_{j+1} of its branch
(the convention that reproduces the variable counts of Table 1).
"""
from __future__ import annotations

import numpy as np


class Tree:
    def __init__(self, parent, prob):
        self.parent = np.asarray(parent, dtype=np.int64)
        self.prob = np.asarray(prob, dtype=np.float64)
        n = len(self.parent)
        self.n = n
        assert self.parent[0] == -1
        stage = np.zeros(n, dtype=np.int64)
        for m in range(1, n):
            assert 0 <= self.parent[m] < m
            stage[m] = stage[self.parent[m]] + 1
        self.stage = stage
        self.horizon = int(stage.max()) + 1
        self.nodes_at = [np.flatnonzero(stage == j) for j in range(self.horizon)]
        self.children = [[] for _ in range(n)]
        for m in range(1, n):
            self.children[self.parent[m]].append(m)
        self.leaves = np.array([m for m in range(n) if not self.children[m]], dtype=np.int64)

    def path(self, m):
        """Nodes from the root down to m (inclusive)."""
        out = []
        while m >= 0:
            out.append(m)
            m = self.parent[m]
        return out[::-1]

    def scenario_paths(self):
        return [self.path(leaf) for leaf in self.leaves]
