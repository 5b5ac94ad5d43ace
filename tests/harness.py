"""Runs the same seeded instance through the oracle and through the C ABI.

The oracle side only uses ``oracle`` and ``synth``; the library side only uses
the binding.  Steps (lambda, preconditioner) are always computed here, on the
oracle side, and passed to the library, so no oracle input comes from the CUDA path.
"""
from __future__ import annotations

from types import SimpleNamespace

import numpy as np

import oracle
import synth


def oracle_build(P):
    tree = oracle.Tree(P["tree"]["parent"], P["tree"]["prob"])
    fac = oracle.factor(P["net"], P["cost"])
    cu = oracle.cost_update(fac, P["cost"], tree, P["alpha2"], P["dhat"], P["eps"], P["q"])
    return tree, fac, cu


def closed_form_steps(fac, tree, lam):
    """Jacobi steps from the closed-form diagonal of the dual Hessian (A = I), times lam."""
    Rinv = np.linalg.inv(fac.R_bar)
    dB = np.einsum("ij,jk,ik->i", fac.B_bar, Rinv, fac.B_bar)
    dL = np.einsum("ij,jk,ik->i", fac.L, Rinv, fac.L)
    cx, cu = np.zeros(tree.n), np.zeros(tree.n)
    for m in range(tree.n):
        path = tree.path(m)
        for i, a in enumerate(path):
            k = len(path) - i
            cx[m] += k * k / (2 * tree.prob[a])
            cu[m] += 1.0 / (2 * tree.prob[a])
    d_s = 1.0 / (cx * dB.mean())
    live = dL > 1e-12 * dL.max()
    dl = np.where(live, dL, dL[live].mean())
    d_p = 1.0 / (cu[:, None] * dl[None, :])
    return {"s": lam * d_s, "z": lam * d_s, "p": lam * d_p}


def oracle_power_lambda(fac, tree, steps_unit, iters=60, seed=0):
    """1 / (largest eigenvalue of D^1/2 H_D D^1/2) by power iteration with Algorithm 1."""
    n, n_x, n_u, n_v = tree.n, fac.n_x, fac.n_u, fac.n_v
    zero = SimpleNamespace(beta=np.zeros((n, n_v)), u_hat=np.zeros((n, n_u)), e=np.zeros((n, n_x)))
    ds, dz, dp = np.sqrt(steps_unit["s"]), np.sqrt(steps_unit["z"]), np.sqrt(steps_unit["p"])
    rng = np.random.default_rng(seed)
    v = [rng.standard_normal((n, n_x)), rng.standard_normal((n, n_x)), rng.standard_normal((n, n_u))]
    lam = 0.0
    for _ in range(iters):
        nrm = np.sqrt(sum((a * a).sum() for a in v))
        v = [a / nrm for a in v]
        x, u = oracle.solve_step(fac, tree, zero, ds[:, None] * v[0], dz[:, None] * v[1], dp * v[2], np.zeros(n_x))
        w = [-ds[:, None] * x, -dz[:, None] * x, -dp * u]
        lam = sum((a * b).sum() for a, b in zip(v, w))
        v = w
    return lam


def full_size_steps(P, power_iters=40):
    """Steps computed on the oracle side without a dense Hessian: the closed-form Jacobi
    diagonal and lambda = 1 / (1.02 L), L from a power iteration of Algorithm 1."""
    tree, fac, _ = oracle_build(P)
    unit = closed_form_steps(fac, tree, 1.0)
    lam = 1.0 / (1.02 * oracle_power_lambda(fac, tree, unit, iters=power_iters))
    return closed_form_steps(fac, tree, lam)


def coupling_residual(P, u):
    """max |E u_n + E_d d_n| over the nodes (the demand coupling of eq. demand-control)."""
    if P["net"]["E"].shape[0] == 0:  # no junction: nothing couples the inputs
        return 0.0
    d = P["dhat"][P["tree"]["stage"]] + P["eps"]
    return float(np.abs(u @ P["net"]["E"].T + d @ P["net"]["Ed"].T).max())


def oracle_run(P, steps, iters, y0=None):
    tree, fac, cu = oracle_build(P)
    return oracle.apg(fac, tree, cu, P["cost"], P["p"], steps, iters, y0=y0)


def stack_y(y3):
    return np.concatenate([y3[0], y3[1], y3[2]], axis=1)


def relerr(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.abs(a - b).max() / (1.0 + np.abs(b).max()))


class Gpu:
    """One instance on the GPU through the C ABI."""

    def __init__(self, P, steps=None, precision=0, precondition=1, lam=0.0, power_iters=0, lambda_margin=0.0,
                 schedule=0, shared_packs=0, tc_width=0):
        import torch

        import paper_1604_01074_gb300 as smpc
        self.smpc, self.torch, self.P = smpc, torch, P
        t = P["tree"]
        self.n = len(t["parent"])
        net, cost = P["net"], P["cost"]
        self.n_x, self.n_u = net["n_x"], net["n_u"]
        self.tree = smpc.smpc_tree_create(t["parent"], t["prob"])
        self.fac = smpc.smpc_factor(self.tree, net, cost, precision=precision, precondition=precondition, lam=lam,
                                    power_iters=power_iters, lambda_margin=lambda_margin, steps=steps,
                                    schedule=schedule, shared_packs=shared_packs, tc_width=tc_width)
        dt = torch.float64 if precision == 0 else torch.float32
        dev = torch.device("cuda", 0)
        self.u = torch.zeros((self.n, self.n_u), dtype=dt, device=dev)
        self.x = torch.zeros((self.n, self.n_x), dtype=dt, device=dev)
        self.y = torch.zeros((self.n, 2 * self.n_x + self.n_u), dtype=dt, device=dev)

    def solve(self, iters, tol=0.0, warm=0, eps=True, check_every=0, ergodic=0, use_graph=0):
        """ergodic=1: the ergodic averages land in self.ubar, self.xbar."""
        P = self.P
        hist = np.zeros((iters, 3))
        u0 = np.zeros(self.smpc.smpc_tree_info_get(self.tree)["n_trees"] * self.n_u)
        if ergodic:
            self.ubar = self.torch.full_like(self.u, float("nan"))
            self.xbar = self.torch.full_like(self.x, float("nan"))
        info = self.smpc.smpc_solve(self.fac, P["p"], P["q"], P["dhat"], P["alpha2"], eps=P["eps"] if eps else None,
                                    max_iters=iters, tol=tol, warm_start=warm, check_every=check_every, sync=1,
                                    u=self.u, x=self.x, y=self.y, u0_host=u0, history_host=hist,
                                    ergodic=ergodic, use_graph=use_graph,
                                    ubar=self.ubar if ergodic else None, xbar=self.xbar if ergodic else None)
        info["history"] = hist[:max(info["iterations"], 0)]
        info["u0"] = u0
        return info

    def arrays(self):
        return self.u.double().cpu().numpy(), self.x.double().cpu().numpy(), self.y.double().cpu().numpy()

    def bars(self):
        return self.ubar.double().cpu().numpy(), self.xbar.double().cpu().numpy()

    def steps(self):
        return self.smpc.smpc_factor_steps(self.fac, self.n, self.n_u)

    def close(self):
        self.smpc.smpc_factor_destroy(self.fac)
        self.smpc.smpc_tree_destroy(self.tree)


def tiny_steps(P):
    tree, fac, _ = oracle_build(P)
    return oracle.jacobi_steps(fac, tree)


def edge_instances():
    """Ragged and degenerate trees: single node, single chain, chains of mixed
    length under non-leaf segments, wide fan-out, random probabilities."""
    out = {
        "single_node": synth.custom(11, 2, 4, 2, 1, synth.make_tree([1], 1)),
        "chain": synth.custom(12, 3, 5, 3, 1, synth.make_tree([1], 7)),
        "root_fan": synth.custom(13, 3, 5, 3, 1, synth.make_tree([9], 3)),
        "late_branch": synth.custom(14, 2, 4, 2, 1, {**synth.tree_from_fanouts_dict([[1], [1], [3], [1, 1, 1], [2, 1, 2]])}),
        "random_a": synth.random_instance(21, horizon=6, max_children=3),
        "random_b": synth.random_instance(22, n_x=4, n_u=7, n_d=4, n_e=2, horizon=5, max_children=4),
        "no_junction": synth.custom(15, 2, 3, 2, 0, synth.make_tree([2, 2], 4)),
    }
    return out
