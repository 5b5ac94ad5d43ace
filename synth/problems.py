"""Seeded SMPC problem instances: network + costs + scenario tree + per-step data.

Workloads (all synthetic; the Barcelona network data and its demand forecasts are
not available, so networks with the paper's dimensions stand in for it, Sec. V):

* ``tiny``: 4 tanks (A = I), 6 actuators with a +-1 incidence B, 3 demands,
  1 junction; horizon 4, branching [2, 2, 2, 1] -> 8 equiprobable scenarios,
  15 nodes; forecast 1 + 0.3 sin(2 pi t / 24); day/night price 2/1 on every
  actuator; W_alpha = 1, W_u = I, W_x = 10, gamma_d = 100; x in [0, 10],
  x_s = 3, u in [0, 2] (a junction supply is widened if needed for feasibility),
  p = 5, q = 1.
* ``barcelona``: n_x = 63, n_u = 114, n_d = 88, n_e = 17 (Sec. V), hourly
  steps (dt = 3600 s), horizon 24, branching [5, 5, 2, 2] -> 100 scenarios,
  2081 nodes; capacities U[500, 5000] m^3, safety level 30 % of capacity,
  u_max U[0.5, 5] m^3/s; demand bases U[0.01, 0.1] m^3/s on a 24 h sinusoid
  with 10 % Gaussian node deviations; the paper's weights W_alpha = 2e4,
  W_u = 1e5 I, W_x = 1e7, gamma_d = 5e7 (Sec. V-B).
* ``large``: the same network with branching [10, 10, 10] -> 1000 scenarios,
  21 111 nodes.
"""
from __future__ import annotations

import numpy as np

from .networks import demand_forecast, make_network, make_tiny_network, node_deviations
from .trees import make_tree, random_tree


def day_night_price(horizon, t0=0, day=2.0, night=1.0):
    t = (t0 + np.arange(horizon)) % 24
    return np.where((t >= 8) & (t < 20), day, night)


def _feasible_input(net, d):
    """Dedicated junction supplies carry the junction demand, all else zero."""
    u = np.zeros(net["n_u"])
    for j in range(net["n_e"]):
        u[j] = d[net["demand_at"] == net["n_x"] + j].sum()
    return u


def assemble(net, tree, rng, W_alpha, W_u, W_x, gamma_d, alpha1, pump_coef, t0=0,
             safety_frac=0.3, p=None, q=None, name="custom"):
    N = tree["horizon"]
    n_x, n_u = net["n_x"], net["n_u"]
    price = day_night_price(N, t0)
    alpha2 = price[:, None] * pump_coef[None, :]
    dhat = demand_forecast(net, N, t0)
    eps = node_deviations(rng, net, dhat, tree["stage"])
    cap = net["cap"]
    if p is None:
        p = rng.uniform(0.4, 0.8, size=n_x) * cap
    if q is None:
        q = _feasible_input(net, dhat[0])
    cost = {
        "W_alpha": float(W_alpha), "alpha1": np.asarray(alpha1, float),
        "W_u": np.asarray(W_u, float), "W_x": float(W_x), "gamma_d": float(gamma_d),
        "x_min": np.zeros(n_x), "x_max": cap.copy(), "x_s": safety_frac * cap,
        "u_min": net["u_min"].copy(), "u_max": net["u_max"].copy(),
    }
    return {"name": name, "net": net, "cost": cost, "tree": tree, "alpha2": alpha2,
            "p": np.asarray(p, float), "q": np.asarray(q, float), "dhat": dhat, "eps": eps}


def tiny(seed=0):
    rng = np.random.default_rng(seed)
    net = make_tiny_network(rng)
    tree = make_tree([2, 2, 2, 1], 4)
    n_u = net["n_u"]
    return assemble(net, tree, rng, W_alpha=1.0, W_u=np.eye(n_u), W_x=10.0, gamma_d=100.0,
                    alpha1=np.zeros(n_u), pump_coef=np.ones(n_u), p=np.full(net["n_x"], 5.0),
                    q=np.ones(n_u), name="tiny")


def barcelona_network(rng):
    return make_network(rng, n_x=63, n_u=114, n_d=88, n_e=17)


def _barcelona_costs(rng, net):
    n_u = net["n_u"]
    alpha1 = np.where(net["actuator_src"] < 0, rng.uniform(0.02, 0.1, size=n_u), 0.0)
    pump = rng.random(n_u) < 0.6
    pump_coef = np.where(pump, rng.uniform(0.01, 0.05, size=n_u), 0.0)
    return alpha1, pump_coef


def barcelona(seed=0, branching=(5, 5, 2, 2), n_scenarios=100, horizon=24, name="barcelona"):
    rng = np.random.default_rng(seed)
    net = barcelona_network(rng)
    alpha1, pump_coef = _barcelona_costs(rng, net)
    tree = make_tree(list(branching), horizon, n_scenarios)
    return assemble(net, tree, rng, W_alpha=2e4, W_u=1e5 * np.eye(net["n_u"]), W_x=1e7,
                    gamma_d=5e7, alpha1=alpha1, pump_coef=pump_coef, name=name)


def large(seed=0):
    return barcelona(seed, branching=(10, 10, 10), n_scenarios=1000, name="large")


def custom(seed, n_x, n_u, n_d, n_e, tree, dt=1.0, weights=(1.0, 1.0, 10.0, 100.0)):
    """Small random instance on a given tree (used for edge cases and brute force)."""
    rng = np.random.default_rng(seed)
    net = make_network(rng, n_x=n_x, n_u=n_u, n_d=n_d, n_e=n_e, dt=dt, cap_range=(10.0, 10.0),
                       umax_range=(1.0, 3.0), demand_base=(0.5, 1.0))
    W_alpha, w_u, W_x, gamma_d = weights
    M = rng.standard_normal((n_u, n_u))
    W_u = w_u * (np.eye(n_u) + 0.2 * (M @ M.T) / n_u)   # SPD, not diagonal
    alpha1 = rng.uniform(0.0, 0.5, size=n_u)
    pump_coef = rng.uniform(0.0, 1.0, size=n_u)
    return assemble(net, tree, rng, W_alpha=W_alpha, W_u=W_u, W_x=W_x, gamma_d=gamma_d,
                    alpha1=alpha1, pump_coef=pump_coef, p=rng.uniform(2.0, 8.0, size=n_x),
                    name="custom")


def general_dynamics(P, seed=0, leak=0.05, exchange=0.03):
    """A copy of instance P whose state matrix is not the identity: tanks that lose a
    fraction of their volume per step and exchange water with the others,
    A = (1 - leak) I + exchange R with R random, zero diagonal and rows summing to one
    (so every row of A sums to 1 - leak + exchange and the dynamics stay bounded)."""
    rng = np.random.default_rng(9000 + seed)
    n_x = P["net"]["n_x"]
    R = rng.uniform(0.0, 1.0, size=(n_x, n_x))
    np.fill_diagonal(R, 0.0)
    if n_x > 1:
        R /= R.sum(axis=1, keepdims=True)
    A = (1.0 - leak) * np.eye(n_x) + exchange * R
    Q = dict(P)
    Q["net"] = {**P["net"], "A": A}
    return Q


def random_instance(seed, n_x=3, n_u=5, n_d=3, n_e=1, horizon=5, max_children=3):
    rng = np.random.default_rng(seed + 1000)
    tree = random_tree(rng, horizon, max_children=max_children)
    return custom(seed, n_x, n_u, n_d, n_e, tree)


BATCH_NETWORKS = ((20, 40), (35, 65), (50, 90), (63, 114))


def batch_network(k, seed=0):
    """Network k (0..3) of the batched workload: n_d ~ 1.4 n_x, n_e ~ 0.15 n_u."""
    n_x, n_u = BATCH_NETWORKS[k]
    rng = np.random.default_rng(7000 + 31 * seed + k)
    net = make_network(rng, n_x=n_x, n_u=n_u, n_d=int(round(1.4 * n_x)), n_e=int(round(0.15 * n_u)))
    return net, rng


def batch_instances(seed=0, count=64):
    """Uneven trees on four shared networks: instance i uses network i % 4, a horizon
    drawn from {12, 18, 24} and a scenario count uniform in [10, 500]; the tree branches
    at stages 0-2 with fan-out ceil(S^(1/3)) and a near-even last branching stage that
    reaches exactly S scenarios.  Barcelona-scale weights; per-instance state,
    forecasts and deviations."""
    nets = [batch_network(k, seed) for k in range(len(BATCH_NETWORKS))]
    costs = [_barcelona_costs(rng, net) for net, rng in nets]
    rng = np.random.default_rng(9000 + seed)
    out = []
    for i in range(count):
        k = i % len(nets)
        net = nets[k][0]
        N = int(rng.choice([12, 18, 24]))
        S = int(rng.integers(10, 501))
        b = 1
        while b ** 3 < S:
            b += 1
        tree = make_tree([b, b, b], N, S)
        alpha1, pump_coef = costs[k]
        P = assemble(net, tree, np.random.default_rng(10000 + 97 * seed + i), W_alpha=2e4,
                     W_u=1e5 * np.eye(net["n_u"]), W_x=1e7, gamma_d=5e7, alpha1=alpha1, pump_coef=pump_coef,
                     t0=int(rng.integers(0, 24)), name=f"batch{i}")
        P["network"] = k
        out.append(P)
    return out


def forest_members(seed, count, n_x=3, n_u=5, n_d=3, n_e=1, max_horizon=6, max_children=3):
    """`count` problems on one network and one cost: uneven random trees (horizons
    3..max_horizon) with their own states, forecasts, prices and deviations."""
    base = custom(seed, n_x, n_u, n_d, n_e, random_tree(np.random.default_rng(seed), 3, max_children))
    rng = np.random.default_rng(20000 + seed)
    out = []
    for i in range(count):
        N = int(rng.integers(3, max_horizon + 1))
        tree = random_tree(np.random.default_rng(30000 + 31 * seed + i), N, max_children=max_children)
        r = np.random.default_rng(40000 + 31 * seed + i)
        P = assemble(base["net"], tree, r, W_alpha=base["cost"]["W_alpha"], W_u=base["cost"]["W_u"],
                     W_x=base["cost"]["W_x"], gamma_d=base["cost"]["gamma_d"], alpha1=base["cost"]["alpha1"],
                     pump_coef=base["alpha2"][0] / day_night_price(3)[0], t0=int(r.integers(0, 24)),
                     p=r.uniform(2.0, 8.0, size=n_x), name=f"member{i}")
        P["cost"] = base["cost"]
        out.append(P)
    return out


def forest(problems):
    """Stacks problems on one network into one forest problem: nodes in breadth-first
    order over all trees (stage 0 holds the roots, tree after tree), per-tree step data
    stacked tree after tree.  members[r][k] is the forest index of node k of tree r."""
    R = len(problems)
    trees = [P["tree"] for P in problems]
    stages = [np.asarray(t["stage"]) for t in trees]
    H = max(int(s.max()) + 1 for s in stages)
    members = [np.zeros(len(t["parent"]), dtype=np.int64) for t in trees]
    order = []
    for j in range(H):
        for r in range(R):
            for k in np.nonzero(stages[r] == j)[0]:
                members[r][k] = len(order)
                order.append((r, int(k)))
    n = len(order)
    parent = np.full(n, -1, dtype=np.int32)
    prob = np.zeros(n)
    stage = np.zeros(n, dtype=np.int64)
    for m, (r, k) in enumerate(order):
        pk = trees[r]["parent"][k]
        parent[m] = -1 if pk < 0 else members[r][pk]
        prob[m] = trees[r]["prob"][k]
        stage[m] = stages[r][k]
    n_d = problems[0]["net"]["n_d"]
    eps = np.zeros((n, n_d))
    for r, P in enumerate(problems):
        eps[members[r]] = P["eps"]
    out = {"name": "forest", "net": problems[0]["net"], "cost": problems[0]["cost"],
           "tree": {"parent": parent, "prob": prob, "stage": stage, "horizon": H},
           "p": np.concatenate([P["p"] for P in problems]), "q": np.concatenate([P["q"] for P in problems]),
           "dhat": np.concatenate([P["dhat"] for P in problems]),
           "alpha2": np.concatenate([P["alpha2"] for P in problems]), "eps": eps,
           "members": members}
    return out
