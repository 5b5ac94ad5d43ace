"""Seeded flow-based water networks shaped like the paper's model (Sec. II).

Tanks hold volumes x (n_x), actuators are pumps/valves moving flow u (n_u) between
an external source, tanks and junctions, demands d (n_d) draw water from tanks or
junctions.  Mass balance gives x+ = A x + B u + G_d d with A = I, and the junction
balances give the coupling E u + E_d d = 0 (eqs. model and demand-control).

Feasibility of the hard coupling with the hard input box (which the paper assumes)
is guaranteed by construction: every junction has a dedicated supply actuator
from an external source whose upper bound is at least ``supply_margin`` (>= 1) times
the largest total demand the generator can draw at that junction, and every lower
bound is zero, so "dedicated supply = junction demand, everything else touching the
junction = 0" is always a feasible input.  E contains an identity block on those supplies, hence full row rank.

Nothing here computes any part of the solver; it only draws data.
"""
from __future__ import annotations

import numpy as np


def make_network(rng, n_x, n_u, n_d, n_e, dt=3600.0, cap_range=(500.0, 5000.0),
                 umax_range=(0.5, 5.0), demand_base=(0.01, 0.1), demand_amp=0.3,
                 demand_sigma=0.1, supply_margin=2.0):
    """Random network; returns dict of FP64 arrays and layout metadata."""
    if n_u < n_x + n_e:
        raise ValueError("need at least one supply actuator per tank and per junction")
    if n_d < n_e:
        raise ValueError("need at least one demand per junction")
    # node ids: tanks 0..n_x-1, junctions n_x..n_x+n_e-1, external source = -1
    src, dst = [], []
    for j in range(n_e):            # dedicated junction supplies (feasibility)
        src.append(-1)
        dst.append(n_x + j)
    for t in range(n_x):            # one supply into every tank, from a source or a junction
        if n_e > 0 and rng.random() < 0.5:
            src.append(n_x + int(rng.integers(n_e)))
        else:
            src.append(-1)
        dst.append(t)
    while len(src) < n_u:            # extra links tank->tank, tank->junction, junction->tank
        kind = rng.integers(3)
        if kind == 0 or n_e == 0:
            a, b = rng.choice(n_x, size=2, replace=False) if n_x > 1 else (0, 0)
            if a == b:
                src.append(-1); dst.append(int(a)); continue
            src.append(int(a)); dst.append(int(b))
        elif kind == 1:
            src.append(int(rng.integers(n_x))); dst.append(n_x + int(rng.integers(n_e)))
        else:
            src.append(n_x + int(rng.integers(n_e))); dst.append(int(rng.integers(n_x)))
    src = np.asarray(src); dst = np.asarray(dst)

    B = np.zeros((n_x, n_u)); E = np.zeros((n_e, n_u))
    for a in range(n_u):
        for node, sign in ((dst[a], 1.0), (src[a], -1.0)):
            if node < 0:
                continue
            if node < n_x:
                B[node, a] += sign * dt
            else:
                E[node - n_x, a] += sign
    # demands: the first n_e sit on the junctions, the rest on random tanks/junctions
    d_at = [n_x + j for j in range(n_e)]
    for _ in range(n_d - n_e):
        if n_e > 0 and rng.random() < 0.2:
            d_at.append(n_x + int(rng.integers(n_e)))
        else:
            d_at.append(int(rng.integers(n_x)))
    d_at = np.asarray(d_at)
    Gd = np.zeros((n_x, n_d)); Ed = np.zeros((n_e, n_d))
    for i, node in enumerate(d_at):
        if node < n_x:
            Gd[node, i] = -dt
        else:
            Ed[node - n_x, i] = -1.0

    base = rng.uniform(*demand_base, size=n_d)
    cap = rng.uniform(*cap_range, size=n_x)
    u_max = rng.uniform(*umax_range, size=n_u)
    # worst demand the generator can draw: base*(1+amp)*(1+3 sigma)
    worst = base * (1.0 + demand_amp) * (1.0 + 3.0 * demand_sigma)
    for j in range(n_e):
        need = worst[d_at == n_x + j].sum()
        u_max[j] = max(u_max[j], supply_margin * need)
    return {
        "n_x": n_x, "n_u": n_u, "n_d": n_d, "n_e": n_e,
        "A": np.eye(n_x), "B": B, "Gd": Gd, "E": E, "Ed": Ed,
        "cap": cap, "u_min": np.zeros(n_u), "u_max": u_max,
        "demand_base": base, "demand_amp": demand_amp, "demand_sigma": demand_sigma,
        "actuator_src": src, "actuator_dst": dst, "demand_at": d_at,
        "supply_of_junction": np.arange(n_e), "dt": dt,
    }


def make_tiny_network(rng):
    """4 tanks, 6 actuators, 3 demands, 1 junction; unit time step (B is a +-1 incidence)."""
    net = make_network(rng, n_x=4, n_u=6, n_d=3, n_e=1, dt=1.0, cap_range=(10.0, 10.0),
                       umax_range=(2.0, 2.0), demand_base=(1.0, 1.0), supply_margin=1.0)
    return net


def demand_forecast(net, horizon, t0=0):
    """Nominal forecast d_hat[j] = base * (1 + amp sin(2 pi (t0+j)/24)) (24 h profile)."""
    t = t0 + np.arange(horizon)
    prof = 1.0 + net["demand_amp"] * np.sin(2.0 * np.pi * t / 24.0)
    return prof[:, None] * net["demand_base"][None, :]


def node_deviations(rng, net, dhat, stage):
    """Per-node forecast errors eps_n ~ N(0, (sigma d_hat)^2), truncated at 3 sigma."""
    sd = net["demand_sigma"] * dhat[stage]
    z = np.clip(rng.standard_normal(sd.shape), -3.0, 3.0)
    return z * sd
