"""A CPU stand-in for one GPU's shard (test infrastructure): the phases of smpc_shard_*
in float64 numpy, with the oracle's factor, cost update and prox as building blocks, so
that the host loop of paper_1604_01074_gb300.shard (the exchange between ranks) runs on
CPU-only gloo ranks.

Chains are the maximal leaf paths (every node on them has at most one child), numbered
by their head's index; the rest of the tree (the top) is replicated.  Per iteration nu:
  local: forward sweep (v_n = v_pi + delta_n, u_n = L v_n + u_hat_n, x_n = x_pi + B_bar v_n
         + e_n) and prox of iteration nu - 1 on this rank's nodes, the dual update and
         w^nu; the backward sweep (Algorithm 1 in the Lambda r form) along its chains; the
         heads' (s, r) summed per cut parent into `exchange`;
  top:   the backward sweep of the top nodes, bottom-up, the cut parents taking the
         exchanged totals for their chain children.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle
from oracle.apg import theta_sequence


def chains_of(parent):
    parent = np.asarray(parent)
    n = len(parent)
    kids = [[] for _ in range(n)]
    for m in range(1, n):
        kids[parent[m]].append(m)
    in_chain = np.zeros(n, bool)
    for m in range(n - 1, -1, -1):  # children have larger indices
        in_chain[m] = len(kids[m]) == 0 or (len(kids[m]) == 1 and in_chain[kids[m][0]])
    heads = [m for m in range(n) if in_chain[m] and (parent[m] < 0 or not in_chain[parent[m]])]
    chains = []
    for h in heads:
        c = [h]
        while kids[c[-1]]:
            c.append(kids[c[-1]][0])
        chains.append(c)
    return chains, [m for m in range(n) if not in_chain[m]], kids


class CpuShard:
    def __init__(self, P, steps, chain_begin, chain_end):
        self.P = P
        t = P["tree"]
        self.tree = oracle.Tree(t["parent"], t["prob"])
        self.fac = oracle.factor(P["net"], P["cost"])
        self.chains, self.top_nodes, self.kids = chains_of(t["parent"])
        self.local_chains = self.chains[chain_begin:chain_end]
        self.cut = sorted({self.tree.parent[c[0]] for c in self.chains})
        self.cut_index = {p: j for j, p in enumerate(self.cut)}
        self.in_chain = np.ones(self.tree.n, bool)
        self.in_chain[self.top_nodes] = False
        self.nodes = sorted(self.top_nodes + [m for c in self.local_chains for m in c])
        n, n_u = self.tree.n, self.fac.n_u
        self.ls = np.asarray(steps["s"], float).reshape(n)
        self.lz = np.asarray(steps["z"], float).reshape(n)
        self.lp = np.broadcast_to(np.asarray(steps["p"], float), (n, n_u)).copy()
        self.width = self.fac.n_x + self.fac.n_v
        self.exchange = torch.zeros((len(self.cut), self.width), dtype=torch.float64)
        self.residuals = None

    # ------------------------------------------------------------------ phases
    def begin(self, step, max_iters, tol):
        P, fac, tree = self.P, self.fac, self.tree
        self.cu = oracle.cost_update(fac, P["cost"], tree, step["alpha2"], step["dhat"], step["eps"], step["q"])
        self.p0 = np.asarray(step["p"], float)
        n, n_x, n_u, n_v = tree.n, fac.n_x, fac.n_u, fac.n_v
        self.y = [np.zeros((n, 2 * n_x + n_u)), np.zeros((n, 2 * n_x + n_u))]  # y^nu, y^{nu-1}
        self.w = np.zeros((n, 2 * n_x + n_u))
        self.delta = np.zeros((n, n_v))
        self.s = np.zeros((n, n_x))
        self.r = np.zeros((n, n_v))
        self.x = np.zeros((n, n_x))
        self.u = np.zeros((n, n_u))
        self.theta = theta_sequence(max_iters + 2)
        self.tol = tol
        self.done = -1
        self.residuals = torch.zeros(3 * (max_iters + 2), dtype=torch.int64)

    def _res(self, k):
        v = self.residuals[3 * k:3 * k + 3].numpy().view(np.float64)
        return v[0] / (1.0 + max(v[1], v[2]))

    def _stopped(self, nu):
        if self.done >= 0:
            return True
        if self.tol > 0 and nu >= 2 and self._res(nu - 2) <= self.tol:
            self.done = nu - 1
            return True
        return False

    def _forward_prox(self, nu):
        """Forward sweep and prox of iteration nu - 1 on this rank's nodes; y^nu, w^nu."""
        fac, cu, cost = self.fac, self.cu, self.P["cost"]
        n_x = fac.n_x
        v = {}
        for m in self.nodes:  # parents first (breadth-first order)
            p = self.tree.parent[m]
            v[m] = (v[p] if p >= 0 else 0.0) + self.delta[m]
            xp = self.x[p] if p >= 0 else self.p0
            self.u[m] = fac.L @ v[m] + cu.u_hat[m]
            self.x[m] = xp + fac.B_bar @ v[m] + cu.e[m]
        S = np.asarray(self.nodes)
        w = self.w[S]
        x, u = self.x[S], self.u[S]
        ls, lz, lp = self.ls[S], self.lz[S], self.lp[S]
        mu = self.tree.prob[S] * cost["W_x"]
        t_s, t_z, t_p = oracle.prox_g(w[:, :n_x] / ls[:, None] + x, w[:, n_x:2 * n_x] / lz[:, None] + x,
                                      w[:, 2 * n_x:] / lp + u, cost, mu, ls, lz)
        ynew = np.concatenate([w[:, :n_x] + ls[:, None] * (x - t_s), w[:, n_x:2 * n_x] + lz[:, None] * (x - t_z),
                               w[:, 2 * n_x:] + lp * (u - t_p)], axis=1)
        res = max(np.abs(x - t_s).max(), np.abs(x - t_z).max(), np.abs(u - t_p).max())
        hz = max(np.abs(x).max(), np.abs(u).max())
        tt = max(np.abs(t_s).max(), np.abs(t_z).max(), np.abs(t_p).max())
        self.residuals[3 * (nu - 1):3 * nu] = torch.from_numpy(np.array([res, hz, tt]).view(np.int64))
        self.y[1][S] = self.y[0][S]
        self.y[0][S] = ynew
        c = self.theta[nu + 1] * (1.0 / self.theta[nu] - 1.0)
        self.w[S] = self.y[0][S] + c * (self.y[0][S] - self.y[1][S])

    def _backward_node(self, m, s_children, r_children):
        fac, n_x = self.fac, self.fac.n_x
        xi = self.w[m, :n_x] + self.w[m, n_x:2 * n_x]
        psi = self.w[m, 2 * n_x:]
        self.s[m] = xi + s_children
        self.r[m] = self.cu.beta[m] + r_children + fac.B_bar.T @ self.s[m] + fac.L.T @ psi
        self.delta[m] = fac.Lam @ self.r[m] / (2.0 * self.tree.prob[m])

    def local(self, nu):
        if self._stopped(nu):
            return
        if nu >= 1:
            self._forward_prox(nu)
        else:
            S = np.asarray(self.nodes)
            self.w[S] = self.y[0][S]
        for c in self.local_chains:
            for k in range(len(c) - 1, -1, -1):
                m = c[k]
                below = c[k + 1] if k + 1 < len(c) else None
                self._backward_node(m, self.s[below] if below is not None else 0.0,
                                    self.r[below] if below is not None else 0.0)
        ex = np.zeros((len(self.cut), self.width))
        for c in self.local_chains:
            j = self.cut_index[self.tree.parent[c[0]]]
            ex[j, :self.fac.n_x] += self.s[c[0]]
            ex[j, self.fac.n_x:] += self.r[c[0]]
        self.exchange.copy_(torch.from_numpy(ex))

    def top(self, nu):
        if self.done >= 0:
            return
        ex = self.exchange.numpy()
        for m in sorted(self.top_nodes, reverse=True):  # children before parents
            s_c = np.zeros(self.fac.n_x)
            r_c = np.zeros(self.fac.n_v)
            for c in self.kids[m]:
                if not self.in_chain[c]:
                    s_c += self.s[c]
                    r_c += self.r[c]
            if m in self.cut_index:
                s_c += ex[self.cut_index[m], :self.fac.n_x]
                r_c += ex[self.cut_index[m], self.fac.n_x:]
            self._backward_node(m, s_c, r_c)

    def tail(self, n):
        if not self._stopped(n) and n >= 1:
            self._forward_prox(n)

    def flags(self):
        return self.done, 0

    def finish(self, launched):
        it = self.done if self.done >= 0 else launched
        v = self.residuals[3 * (it - 1):3 * it].numpy().view(np.float64)
        return {"iterations": it, "rho": float(v[0]), "rho_rel": float(v[0] / (1.0 + max(v[1], v[2])))}
