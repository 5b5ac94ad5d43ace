"""The closed-loop key performance indicators of Sec. V, as bench.py --serve reports them,
and the serving harness that records the closed loops they are computed from (driven here
by a stand-in for the library's server, on the CPU)."""
import types

import numpy as np

import bench
import synth


def test_kpis_by_hand():
    u = np.array([[1.0, -2.0], [3.0, 0.0]])
    x = np.array([[1.0, 5.0], [4.0, 2.0]])
    alpha = np.array([[1.0, 2.0], [0.5, 1.0]])
    k = bench.closed_loop_kpis(u, x, alpha, np.zeros(2), np.array([2.0, 3.0]))
    assert k["steps"] == 2
    assert abs(k["KPI_E"] - (1 * 1 + 2 * 2 + 0.5 * 3 + 1 * 0) / 2) < 1e-15           # 3.25
    assert abs(k["KPI_dU"] - ((1 + 4) + (4 + 4)) / 2) < 1e-15                        # 6.5
    assert abs(k["KPI_S"] - (1 + 1)) < 1e-15                                        # [1,0] + [0,1]
    assert abs(k["KPI_R_pct"] - 5.0 / 6.0 * 100.0) < 1e-12


class _FakeServer:
    """Completes every request at its first poll with a fixed input u_0 = 0.05 (and counts)."""

    def __init__(self):
        self.next, self.open = 1, {}

    def smpc_submit(self, server, fac, p, q, dhat, alpha2, eps=None, max_iters=0, tol=0.0, warm_start=0,
                    check_every=0):
        assert p.shape == (fac["n_x"],) and alpha2.shape[1] == fac["n_u"]
        t = self.next
        self.next += 1
        self.open[t] = fac["n_u"]
        return t

    def smpc_poll(self, server, ticket, u0_host=None):
        n_u = self.open.pop(ticket)
        u0_host[:] = 0.05 * np.ones(n_u)
        return {"queue_ms": 0.0, "run_ms": 1.0, "iterations": 10, "rho_rel": 5e-4}


def test_serving_harness_records_the_closed_loops():
    sess = []
    for i, P in enumerate((synth.tiny(0), synth.random_instance(22, n_x=4, n_u=7, n_d=4, n_e=2, horizon=5))):
        sess.append({"P": P, "fac": {"n_x": P["net"]["n_x"], "n_u": P["net"]["n_u"]}, "x": P["p"].copy(),
                     "q": P["q"].copy(), "k": 0, "pending": [], "rng": np.random.default_rng(100 + i),
                     "traj": [], "q_start": P["q"].copy()})
    args = types.SimpleNamespace(serve_max_iters=100, tol=1e-3)
    w = bench._serve_window(_FakeServer(), None, sess, 200.0, 0.2, 1.0, args, np.random.default_rng(0))
    assert w["completed"] == w["offered"] > 0 and w["unfinished"] == 0
    assert w["reached_tol"] == w["completed"]
    K = bench.serve_kpis(sess)
    assert K["sessions"] == sum(1 for s_ in sess if s_["traj"])
    for s_ in sess:
        if not s_["traj"]:
            continue
        P = s_["P"]
        # the recorded states follow the plant from the start state with the applied inputs
        x = P["p"].copy()
        rng = np.random.default_rng(100 + sess.index(s_))
        for k, (u0, xk, a) in enumerate(s_["traj"]):
            x = bench._plant_step(P, x, u0, k, rng)
            np.testing.assert_allclose(xk, x, rtol=0, atol=1e-12)
            np.testing.assert_allclose(a, P["cost"]["alpha1"] + bench._session_prices(P, k)[0], rtol=0, atol=0)
        u, xs, al = (np.array([t[i] for t in s_["traj"]]) for i in range(3))
        one = bench.closed_loop_kpis(u, xs, al, s_["q_start"], P["cost"]["x_s"])
        assert K["KPI_E"]["min"] <= one["KPI_E"] <= K["KPI_E"]["max"]
        assert one["KPI_dU"] >= 0 and one["KPI_S"] >= 0 and one["KPI_R_pct"] > 0
