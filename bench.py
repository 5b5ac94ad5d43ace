"""Benchmark: SMPC solves/s to a 1e-3 relative primal-dual residual on the
Barcelona-shaped synthetic network (n_x = 63, n_u = 114, n_d = 88, n_e = 17,
horizon 24).  Default workload: the large tree, branching [10, 10, 10] ->
1000 scenarios, 21 111 nodes, float32 per-node packs; the 2081-node tree
(branching [5, 5, 2, 2], 100 scenarios) runs as a leg.

One step = one SMPC solve: cost update on the device, then APG iterations until
rho_rel <= 1e-3 (or the cap), cold start y^0 = 0, on one MPC step's synthetic
inputs (state, forecast, prices differ from step to step).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun every rank solves its own copy of
the workload (replicas: scaling "weak"); the timed region is bracketed by a
barrier and a device synchronize on both sides and the max time over ranks is used.
Without torchrun, --gpus N > 1 starts N ranks itself (torch.distributed.run).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SMPC solves/sec and ms per solve to 1e-3 primal-dual residual; APG iters/s; p50/p99"
WORKLOADS = {
    "large": "Barcelona-shaped large tree: n_x=63, n_u=114, n_d=88, n_e=17, N=24, branching [10,10,10] -> "
             "1000 scenarios, 21111 nodes",
    "barcelona": "Barcelona-shaped single tree: n_x=63, n_u=114, n_d=88, n_e=17, N=24, branching [5,5,2,2] -> "
                 "100 scenarios, 2081 nodes",
    "tiny": "tiny: 4 tanks, 6 actuators, N=4, branching [2,2,2,1] -> 8 scenarios, 15 nodes",
}
PREC_NAMES = {0: "f64", 1: "f32", 2: "bf16"}
PREC_KEYS = {0: "fp64", 1: "fp32", 2: "bf16"}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# float64 FMA throughput of the GB300, measured live by smpc_fma_peak (the library's
# chain-of-FMA diagnostic); this value is used only when that call fails.
FP64_FMA_TFLOPS = 1.157


def recorded_traffic(prec_name):
    """DRAM bytes per launch from the last ncu capture in profiles/, if the kernel
    source is unchanged since (else None)."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        src = open(os.path.join(ROOT, "paper_1604_01074_gb300", "csrc", "kernels.cu"), "rb").read()
        if hashlib.sha256(src).hexdigest()[:16] != rec.get("kernel_sha256_16"):
            return None
        return rec.get(prec_name, {}).get("dram_bytes_per_launch")
    except Exception:  # noqa: BLE001
        return None


# --------------------------------------------------------------------- workload
def make_problem(config, seed=0):
    import synth
    if config == "tiny":
        return synth.tiny(seed)
    if config == "large":
        return synth.large(seed)
    return synth.barcelona(seed)


def step_inputs(P, k):
    """Inputs of MPC step k: forecast and prices shifted by k hours, state perturbed."""
    import synth
    from synth.problems import day_night_price
    N = P["tree"]["horizon"]
    net = P["net"]
    dhat = synth.demand_forecast(net, N, t0=k)
    price = day_night_price(N, t0=k)
    base = P["alpha2"] / np.maximum(day_night_price(N, 0)[:, None], 1e-300)
    alpha2 = price[:, None] * base
    rng = np.random.default_rng(1000 + k)
    p = P["p"] * (1.0 + 0.02 * rng.standard_normal(P["p"].shape))
    return {"p": p, "q": P["q"], "dhat": dhat, "alpha2": alpha2}


ANCHOR_EVERY = 16  # the library's default anchor interval of bfloat16 solves


def algorithmic_bytes_per_iteration(n, n_x, n_u, n_v, prec):
    """Bytes one APG iteration must move: every pack entry once ([Bbar; L] is read
    once and used for both of its mat-vecs), the node vectors in the vector type and
    the dual state (8 bytes per entry).  bfloat16 solves average one float32-pack
    anchor iteration per ANCHOR_EVERY and read the anchor h and w besides."""
    vs = 8 if prec == 0 else 4
    n_k = n_x + n_u
    nd = 2 * n_x + n_u
    mat = n_k * n_v + n_v * n_v
    if prec == 2:
        ms = (2 * (ANCHOR_EVERY - 1) + 4) / ANCHOR_EVERY
    else:
        ms = {0: 8, 1: 4}[prec]
    # forward+prox reads h, e, u_hat, steps (n_u + 2) and reciprocals (n_u + 2), mu;
    # writes u, x, w.  The dual state: reads y^nu, y^{nu-1}; writes y^{nu+1}.
    # backward reads w, beta; writes h.
    vec_r = n_k + n_x + n_u + 2 * (n_u + 2) + 1 + n_k + n_v
    vec_w = n_k + n_k + n_k
    if prec == 2:
        vec_r += 2 * n_k  # anchor h and w
    state = 3 * nd * 8
    return n * (mat * ms + (vec_r + vec_w) * vs + state), n * mat, n * 2 * (n_k * n_v + n_v * n_v + n_k * n_v)


STAGES = {1: ["apg_iter"], 2: ["fwd_scan", "prox_node", "scan_s", "node_mv_gt", "scan_r", "node_mv_dh"],
          3: ["fwd_scan", "prox_node", "apg_iter_gt", "node_mv_dh"], 4: ["fwd_scan", "prox_node", "apg_iter_bwd"]}


def stage_bytes(stage, n, n_x, n_u, n_v, prec, shared):
    """Algorithmic bytes of one launch of a node-parallel kernel: the matrix entries it
    applies (per node, unless the pack is shared) and its node vectors.  [Bbar; L]' y
    reads [Bbar; L] (n_k x n_v); Lambda r and [Bbar; L] delta read Lambda and [Bbar; L]:
    together the 43,747 entries per node of one iteration (n_x = 63, n_u = 114)."""
    ms = {0: 8, 1: 4, 2: 2}[prec]
    vs = 8 if prec == 0 else 4
    n_k = n_x + n_u
    if stage == "node_mv_gt":
        return n * ((0 if shared else n_k * n_v * ms) + (n_k + n_v) * vs)
    if stage == "apg_iter_gt":
        return n * ((0 if shared else n_k * n_v * ms) + (n_k + n_x + 2 * n_v) * vs)
    if stage == "node_mv_dh":
        return n * ((0 if shared else (n_k * n_v + n_v * n_v) * ms) + (n_v + n_k) * vs)
    if stage == "apg_iter_bwd":
        # the whole backward sweep with each pack read once: [Bbar; L] and Lambda per node;
        # w (n_k) and beta (n_v) in, h (n_k) out, s and r published (n_x + n_v)
        return n * ((0 if shared else (n_k * n_v + n_v * n_v) * ms) + (2 * n_k + n_x + 2 * n_v) * vs)
    return None


def stage_flops(stage, n, n_x, n_u, n_v):
    """Flops of one launch of a pack-reading kernel: 2 per matrix entry applied."""
    n_k = n_x + n_u
    if stage in ("node_mv_gt", "apg_iter_gt"):
        return n * 2 * n_k * n_v
    if stage == "node_mv_dh":
        return n * 2 * (n_k * n_v + n_v * n_v)
    if stage == "apg_iter_bwd":
        return n * 2 * (2 * n_k * n_v + n_v * n_v)
    return None


# --------------------------------------------------------------------- CPU oracle leg
def oracle_sample(config, iters, step=0, start_at=0.0):
    """Times the FP64 oracle (as it stands) for `iters` APG iterations on MPC step
    `step`'s inputs of the workload; JSON to stdout.  With start_at (a wall-clock time),
    the timed part waits for it, so that processes started together time together."""
    import oracle
    P = make_problem(config)
    P.update(step_inputs(P, step))
    tree = oracle.Tree(P["tree"]["parent"], P["tree"]["prob"])
    fac = oracle.factor(P["net"], P["cost"])
    cu = oracle.cost_update(fac, P["cost"], tree, P["alpha2"], P["dhat"], P["eps"], P["q"])
    oracle.apg(fac, tree, cu, P["cost"], P["p"], 1e-9, 2)   # warm caches
    if start_at > 0:
        time.sleep(max(0.0, start_at - time.time()))
    t0 = time.perf_counter()
    oracle.apg(fac, tree, cu, P["cost"], P["p"], 1e-9, iters)
    dt = time.perf_counter() - t0
    print(json.dumps({"ms_per_iter": 1e3 * dt / iters, "iters": iters, "seconds": dt}))


def _oracle_cmd(config, iters, step=0, start_at=0.0):
    return [sys.executable, os.path.abspath(__file__), "--oracle-sample", str(iters), "--config", config,
            "--oracle-step", str(step), "--oracle-start", repr(start_at)]


def _oracle_env(threads=1):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = str(threads)
    env["CUDA_VISIBLE_DEVICES"] = ""
    return env


def run_oracle_sample(config, iters, threads=1, step=0):
    t0 = time.perf_counter()
    r = subprocess.run(_oracle_cmd(config, iters, step), capture_output=True, text=True, env=_oracle_env(threads),
                       cwd=ROOT, timeout=900)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    out = json.loads(r.stdout.strip().splitlines()[-1])
    out["wall_s"] = time.perf_counter() - t0
    return out


def run_oracle_parallel(config, iters, procs, setup_s):
    """`procs` single-threaded oracle processes at once, each on its own MPC step's inputs
    (independent solves, one per host core), timing together from a common start time
    after their set-up; returns their samples and the wall time."""
    t0 = time.perf_counter()
    start_at = time.time() + 2.0 * setup_s + 5.0
    ps = [subprocess.Popen(_oracle_cmd(config, iters, k, start_at), stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                           text=True, env=_oracle_env(1), cwd=ROOT) for k in range(procs)]
    out = []
    for p_ in ps:
        o, e = p_.communicate(timeout=900)
        if p_.returncode != 0:
            raise RuntimeError(e[-2000:])
        out.append(json.loads(o.strip().splitlines()[-1]))
    return out, time.perf_counter() - t0


def oracle_iters_to_tol(config):
    path = os.path.join(ROOT, "tests", "golden", "oracle_iters_to_tol.json")
    if os.path.exists(path):
        d = json.load(open(path))
        if config in d:
            return int(d[config]["iterations"]), d[config]
    return None, None


def cpu_baseline(config, iters_to_tol, seconds=12.0):
    """The FP64 oracle as it stands, timed on the host cores: one process (one core), and
    one process per core on independent step inputs (all cores).  Each times a bounded
    sample of about `seconds` of APG iterations, scaled to the oracle's own iteration
    count to rho_rel <= 1e-3."""
    probe = run_oracle_sample(config, 3)
    n = max(5, min(2000, int(1000.0 * seconds / max(probe["ms_per_iter"], 1e-3))))
    one = run_oracle_sample(config, n)
    cores = os.cpu_count() or 1
    many, wall = run_oracle_parallel(config, n, cores, probe["wall_s"])
    # all cores: each process's own iteration rate, summed (they ran at the same time)
    iters_per_s_all = sum(1000.0 / m["ms_per_iter"] for m in many)
    ms_solve = one["ms_per_iter"] * iters_to_tol
    return {"value": 1000.0 / ms_solve, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"{n} FP64 APG iterations of the same workload timed ({one['seconds']:.1f} s), "
                      f"scaled to {iters_to_tol} iterations per solve (the oracle's own count to 1e-3)",
            "ms_per_iter": one["ms_per_iter"], "iters_per_s": 1000.0 / one["ms_per_iter"],
            "host_cores": cores,
            "all_cores": {"value": iters_per_s_all / iters_to_tol, "unit": "solves/s", "cores": cores,
                          "kind": "oracle", "iters_per_s": iters_per_s_all, "wall_s": wall,
                          "sample": f"{cores} single-threaded oracle processes at once, one per host core, each "
                                    f"{n} FP64 APG iterations of its own MPC step's inputs; summed iteration "
                                    f"rate scaled to {iters_to_tol} iterations per solve"}}


# --------------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, out_path):
        self.path = out_path
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            dev = os.environ.get("LOCAL_RANK", "0")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", dev, f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            rows = []
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for i, nm in enumerate(names):
                    if r[5 + i].strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------- distributed helpers
def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def aggregate(local_units, local_seconds, backend_device=None):
    """Whole-job throughput: units summed over ranks / max time over ranks."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return local_units, local_seconds
    dev = backend_device or torch.device("cpu")
    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=dev)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()), float(t.item())


# --------------------------------------------------------------------- our arm
class Solver:
    def __init__(self, P, precision, device, schedule=0, shared_packs=0, steps=None):
        import torch

        import paper_1604_01074_gb300 as smpc
        self.smpc, self.torch, self.P = smpc, torch, P
        self.use_graph = 0  # smpc_solve_opts.use_graph for this solver's solves
        t, net = P["tree"], P["net"]
        self.n, self.n_x, self.n_u = len(t["parent"]), net["n_x"], net["n_u"]
        self.tree = smpc.smpc_tree_create(t["parent"], t["prob"])
        self.info = smpc.smpc_tree_info_get(self.tree)
        self.fac = smpc.smpc_factor(self.tree, net, P["cost"], precision=precision, precondition=1, schedule=schedule,
                                    shared_packs=shared_packs, steps=steps)
        self.schedule, self.tuned_ms = smpc.smpc_factor_schedule(self.fac)
        dt = torch.float64 if precision == 0 else torch.float32
        self.u = torch.empty((self.n, self.n_u), dtype=dt, device=device)
        self.x = torch.empty((self.n, self.n_x), dtype=dt, device=device)
        self.eps_dev = torch.from_numpy(np.ascontiguousarray(P["eps"])).to(device)
        self.device = device

    def device_inputs(self, inp):
        T = self.torch
        return {k: T.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).to(self.device) for k, v in inp.items()}

    def pinned_inputs(self, inp):
        T = self.torch
        return {k: T.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).pin_memory() for k, v in inp.items()}

    def solve(self, inp, max_iters, tol, stream, eps=True, sync=0, u0=None):
        ptr = lambda t: t.data_ptr() if hasattr(t, "data_ptr") else t  # noqa: E731
        return self._raw_solve(ptr(inp["p"]), ptr(inp["q"]), ptr(inp["dhat"]), ptr(inp["alpha2"]),
                               self.eps_dev.data_ptr() if eps else None, max_iters, tol, stream, sync, u0)

    def _raw_solve(self, p, q, dhat, alpha2, eps, max_iters, tol, stream, sync, u0):
        import ctypes
        smpc = self.smpc
        dp = ctypes.POINTER(ctypes.c_double)
        cast = lambda a: None if a is None else ctypes.cast(ctypes.c_void_p(a), dp)  # noqa: E731
        D = smpc.smpc_step_data(cast(p), cast(q), cast(dhat), cast(eps), cast(alpha2))
        O = smpc.smpc_solve_opts(int(max_iters), float(tol), 0, 64, int(sync), 0, 0, int(self.use_graph))
        R = smpc.smpc_result(self.u.data_ptr(), self.x.data_ptr(), None,
                             None if u0 is None else u0.ctypes.data_as(dp), None, -1, 0.0, 0.0, 0)
        smpc._check(smpc.lib().smpc_solve(self.fac, ctypes.byref(D), ctypes.byref(O), ctypes.byref(R),
                                          stream.cuda_stream), "smpc_solve")
        return {"iterations": R.iterations, "rho_rel": R.rho_rel, "launches": R.launches}

    def finish(self):
        return self.smpc.smpc_solve_info(self.fac)

    def close(self):
        self.smpc.smpc_factor_destroy(self.fac)
        self.smpc.smpc_tree_destroy(self.tree)


def time_per_iteration(S, inp, stream, lo=100, hi=400, reps=3):
    """Average duration of one iteration launch: events around fixed-length solves
    (tol = 0) of two lengths; the difference removes the per-solve fixed cost."""
    torch = S.torch
    out = {}
    for iters in (lo, hi):
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            S.solve(inp, iters, 0.0, stream)
            e1.record(stream)
            e1.synchronize()
            S.finish()
            ts.append(e0.elapsed_time(e1))
        out[iters] = statistics.median(ts)
    return (out[hi] - out[lo]) / (hi - lo)


SCHED_NAMES = {1: "chain", 2: "node-parallel", 3: "hybrid", 4: "fused chain pass"}


def kernel_roofline(S, P, prec, inp, stream, fp64_peak, iters=200):
    """Per-kernel device times of a live profiling solve (CUDA events between the launches,
    smpc_profile_solve) and the roofline of the dominant kernel: algorithmic bytes (or
    flops) per launch / its mean duration."""
    t_iter_ms = time_per_iteration(S, inp, stream, *((20, 60) if prec == 0 else (100, 400)))
    n_v = S.n_u - np.linalg.matrix_rank(P["net"]["E"])
    nbytes, _, flops = algorithmic_bytes_per_iteration(S.n, S.n_x, S.n_u, n_v, prec)
    host = {k: v.cpu().numpy() for k, v in inp.items()}
    stage_ms = S.smpc.smpc_profile_solve(S.fac, host["p"], host["q"], host["dhat"], host["alpha2"], eps=P["eps"],
                                         iters=iters)
    names = STAGES[S.schedule]
    hbm, src = peaks()
    if S.schedule == 1:
        kern, k_ms, k_bytes = "apg_iter", stage_ms[0], nbytes
    else:
        k = int(np.argmax(stage_ms))
        kern, k_ms = names[k], stage_ms[k]
        k_bytes = stage_bytes(kern, S.n, S.n_x, S.n_u, n_v, prec, False)
    if prec == 0:
        k_flops = flops if S.schedule == 1 else stage_flops(kern, S.n, S.n_x, S.n_u, n_v)
        achieved = (k_flops or 0) / (k_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak, "traffic": recorded_traffic("fp64"),
                "peak_source": "float64 FMA throughput measured live by smpc_fma_peak"}
    else:
        achieved = (k_bytes or 0) / (k_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": recorded_traffic(f"{PREC_KEYS[prec]}_{kern}_{S.n}"), "peak_source": f"{src} hbm_gbs"}
    roof.update({"kernel": kern, "us_per_launch": 1000.0 * k_ms, "bytes_per_launch": k_bytes,
                 "timing": f"CUDA events between the launches of a {iters}-iteration profiling solve",
                 "stage_us": {n_: 1000.0 * t for n_, t in zip(names, stage_ms)},
                 "us_per_iteration": 1000.0 * t_iter_ms,
                 "iteration_bytes": nbytes, "iteration_frac_of_hbm": nbytes / (t_iter_ms * 1e-3) / 1e9 / hbm})
    return roof


def timed_solves(S, dev_in, ks, stream, args, flush):
    torch = S.torch
    times, iters, launches = [], [], 0
    for k in ks:
        flush.fill_(float(k))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        S.solve(dev_in[k], args.max_iters, args.tol, stream)
        e1.record(stream)
        info = S.finish()
        times.append(e0.elapsed_time(e1))
        iters.append(info["iterations"])
        launches += info["launches"]
    return times, iters, launches


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    import paper_1604_01074_gb300 as smpc
    device = torch.device("cuda", local_rank)
    torch.cuda.set_device(device)
    if world > 1:
        dist.init_process_group("nccl", device_id=device)
    prec = {"fp64": 0, "fp32": 1, "bf16": 2}[args.precision]
    P = make_problem(args.config, seed=0)
    S = Solver(P, prec, device, args.schedule)
    S.use_graph = 0 if args.no_graph else 1  # the warm-up solves capture the chunks, the timed ones replay them
    stream = torch.cuda.current_stream(device)
    n_steps = args.steps + args.warmup
    inputs = [step_inputs(P, k) for k in range(n_steps)]
    dev_in = [S.device_inputs(i) for i in inputs]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=device)  # 256 MB > L2

    log("factor ready", S.info, "schedule", S.schedule, S.tuned_ms)
    for k in range(args.warmup):  # warm-up solves (untimed)
        S.solve(dev_in[k], args.max_iters, args.tol, stream)
        S.finish()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    fd, clk_path = tempfile.mkstemp(prefix="smpc_clocks_", suffix=".csv")
    os.close(fd)
    clk = ClockSampler(clk_path)
    with clk:
        times, iters, launches = timed_solves(S, dev_in, range(args.warmup, n_steps), stream, args, flush)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = clk.summary()
    os.unlink(clk_path)
    log("timed solves ms", times, "iterations", iters)
    local_s = sum(times) / 1000.0
    units, secs = aggregate(args.steps, local_s, device if world > 1 else None)
    value = units / secs
    ms_per_step = 1000.0 * local_s / args.steps

    try:
        fp64_peak = smpc.smpc_fma_peak(0)
    except Exception:  # noqa: BLE001
        fp64_peak = FP64_FMA_TFLOPS
    roof = kernel_roofline(S, P, prec, dev_in[0], stream, fp64_peak)
    log("roofline", roof)

    # end to end through smpc_solve with host (pinned) inputs and the host read of u_0 and
    # the residual, wall clock; a bounded number of the timed steps' inputs
    n_e2e = max(1, min(args.steps, args.e2e_steps))
    pin_in = [S.pinned_inputs(inputs[k]) for k in range(args.warmup, args.warmup + n_e2e)]
    u0 = np.zeros(S.n_u)
    e2e_t = []
    for k, pin in enumerate(pin_in):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.solve(pin, args.max_iters, args.tol, stream, sync=1, u0=u0)
        e2e_t.append(time.perf_counter() - t0)
    e2e_units, e2e_secs = aggregate(n_e2e, sum(e2e_t), device if world > 1 else None)
    log("e2e s", e2e_t)
    h2d = sum(int(np.asarray(v).nbytes) for v in inputs[0].values())
    d2h = 8 * S.n_u + 8 + 24

    result = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": PREC_NAMES[prec], "data": "synthetic",
        "config": {"workload": WORKLOADS[args.config], "solve": "cold start, tol 1e-3 on rho_rel", "tol": args.tol,
                   "max_iters": args.max_iters, "precision": args.precision, "packs": "per node",
                   "schedule": SCHED_NAMES[S.schedule], "schedule_tuning_ms": S.tuned_ms,
                   "l2": "inputs (packs) larger than L2, and a 256 MB buffer written between timed solves",
                   "parallelism": f"replicas x{world}",
                   "launch": "plain launches" if args.no_graph else
                   "64-iteration chunks as CUDA graphs (smpc_solve use_graph; captured by the warm-up solves)"},
        "iterations_mean": float(np.mean(iters)), "apg_iters_per_s": float(np.sum(iters)) / local_s * world,
        "p50_ms": float(np.percentile(times, 50)), "p99_ms": float(np.percentile(times, 99)),
        "roofline": roof, "clocks": clocks, "gpu_launches": launches,
        "e2e": {"value": e2e_units / e2e_secs, "unit": "solves/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": n_e2e,
                "note": "smpc_solve with pinned host inputs, sync = 1 (u_0 and the residual read back), wall clock"},
        "fp64_fma_tflops": fp64_peak,
        "tree": S.info,
    }
    log("headline", {k: result[k] for k in ("value", "ms_per_step", "iterations_mean", "p50_ms", "p99_ms")})
    S.close()
    if args.other_legs and rank == 0:
        result["legs"] = run_legs(args, P, prec, dev_in, stream, flush, fp64_peak)
    if rank == 0 and not args.no_cpu_baseline:
        it_ref = int(np.mean(iters))
        stored, _ = oracle_iters_to_tol(args.config)
        try:
            result["cpu_baseline"] = cpu_baseline(args.config, stored or it_ref)
            if not stored:
                result["cpu_baseline"]["note"] = "no stored oracle iteration count: scaled by the GPU's count"
            log("cpu baseline", result["cpu_baseline"])
        except Exception as exc:  # noqa: BLE001
            result["cpu_baseline"] = {"error": str(exc)[-300:]}
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return result


def run_legs(args, P, prec, dev_in, stream, flush, fp64_peak):
    """Other precisions and pack layouts on the headline workload (iteration cost and the
    roofline of their dominant kernel), and, for the large tree, the 2081-node tree with
    float32 per-node packs (solves to tol) and every precision's solution at tol against
    the float64 solve at tol there (same steps)."""
    torch = __import__("torch")
    device = torch.device("cuda", torch.cuda.current_device())
    legs = {}
    steps = None  # every precision takes the float64 factor's steps
    n = len(P["tree"]["parent"])
    for other in (0, 1, 2):
        So = Solver(P, other, device, steps=steps)
        try:
            if steps is None:
                steps = So.smpc.smpc_factor_steps(So.fac, n, P["net"]["n_u"])[1]
            if other != prec:
                leg = kernel_roofline(So, P, other, dev_in[0], stream, fp64_peak)
                leg["schedule"] = SCHED_NAMES[So.schedule]
                legs[PREC_NAMES[other] + "_per_node"] = leg
                log("leg", PREC_NAMES[other], {k: leg[k] for k in ("us_per_iteration", "kernel", "frac")})
        finally:
            So.close()
    # shared packs (one pack for all nodes): solves to tol
    Sh = Solver(P, prec, device, shared_packs=1)
    try:
        Sh.use_graph = 1
        times, iters, _ = timed_solves(Sh, dev_in, range(min(len(dev_in), args.leg_solves)), stream, args, flush)
        legs[PREC_NAMES[prec] + "_shared_packs"] = {
            "solves_per_s": 1000.0 * len(times) / sum(times), "ms_per_solve": float(np.mean(times)),
            "iterations_mean": float(np.mean(iters)), "schedule": SCHED_NAMES[Sh.schedule],
            "factor_device_bytes": Sh.smpc.smpc_factor_device_bytes(Sh.fac),
            "note": "one pack per factor: the per-node matrices differ only by 1/(2 p_n), applied to Lambda r"}
        log("leg shared", legs[PREC_NAMES[prec] + "_shared_packs"])
    finally:
        Sh.close()
    if args.config != "large":
        return legs
    Pb = make_problem("barcelona")
    nb = len(Pb["tree"]["parent"])
    Sb = Solver(Pb, 1, device)
    try:
        Sb.use_graph = 1
        inb = [Sb.device_inputs(step_inputs(Pb, k)) for k in range(args.leg_solves + 1)]
        Sb.solve(inb[0], args.max_iters, args.tol, stream)  # warm-up (captures the graphs)
        Sb.finish()
        times, iters, _ = timed_solves(Sb, inb, range(1, args.leg_solves + 1), stream, args, flush)
        leg = {"workload": WORKLOADS["barcelona"], "precision": "fp32", "packs": "per node",
               "solves_per_s": 1000.0 * len(times) / sum(times), "ms_per_solve": float(np.mean(times)),
               "iterations_mean": float(np.mean(iters)), "schedule": SCHED_NAMES[Sb.schedule]}
        leg["roofline"] = kernel_roofline(Sb, Pb, 1, inb[0], stream, fp64_peak)
        legs["barcelona_fp32_per_node"] = leg
        log("leg barcelona", {k: leg[k] for k in ("solves_per_s", "iterations_mean", "schedule")})
    finally:
        Sb.close()
    # every precision's solution at tol against the float64 solution at tol (same steps)
    sols, its, steps_b = {}, {}, None
    for other in (0, 1, 2):
        So = Solver(Pb, other, device, steps=steps_b)
        try:
            if steps_b is None:
                steps_b = So.smpc.smpc_factor_steps(So.fac, nb, Pb["net"]["n_u"])[1]
            inp = So.device_inputs(step_inputs(Pb, 0))
            So.solve(inp, args.max_iters, args.tol, stream)
            its[other] = So.finish()["iterations"]
            sols[other] = (So.u.double().cpu().numpy(), So.x.double().cpu().numpy())
        finally:
            So.close()
    u64, x64 = sols[0]
    d = Pb["dhat"][Pb["tree"]["stage"]] + Pb["eps"]
    legs["error_at_tol_vs_fp64"] = {
        PREC_NAMES[k]: {"u": float(np.abs(u - u64).max() / (1 + np.abs(u64).max())),
                        "x": float(np.abs(x - x64).max() / (1 + np.abs(x64).max())),
                        "coupling": float(np.abs(u @ Pb["net"]["E"].T + d @ Pb["net"]["Ed"].T).max()),
                        "iterations": its[k]}
        for k, (u, x) in sols.items()}
    legs["error_at_tol_vs_fp64"]["workload"] = WORKLOADS["barcelona"]
    legs["error_at_tol_vs_fp64"]["note"] = (
        "each precision solved to rho_rel <= tol with the float64 factor's steps, against the float64 solution at "
        "tol, relative to 1 + max |.|; the -m gpu tests tie every precision to the FP64 oracle element by element")
    log("errors at tol", legs["error_at_tol_vs_fp64"])
    return legs


def profile_solve(args):
    import torch
    device = torch.device("cuda", 0)
    prec = {"fp64": 0, "fp32": 1, "bf16": 2}[args.precision]
    P = make_problem(args.config, seed=0)
    S = Solver(P, prec, device, args.schedule, shared_packs=int(args.shared_packs))
    stream = torch.cuda.current_stream(device)
    inp = S.device_inputs(step_inputs(P, 0))
    # a warm-up solve, then the profiled one inside a profiler range (ncu --profile-from-start off
    # captures only its launches, not the factor's power iteration or schedule tuning)
    S.solve(inp, 20, 0.0, stream)
    S.finish()
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    S.solve(inp, args.profile_solve, 0.0, stream)
    info = S.finish()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    S.close()
    print(json.dumps({"profile_solve": args.profile_solve, "precision": args.precision, "info": info}))


# --------------------------------------------------------------------- serving (closed loop)
SERVE_WORKLOAD = ("64 closed-loop MPC sessions on 4 networks (n_x, n_u) in {(20,40),(35,65),(50,90),(63,114)}, "
                  "N in {12,18,24}, 10-500 scenarios (249,644 nodes in all); Poisson arrivals")


def _session_prices(P, k):
    """The time-varying prices alpha_2 of MPC step k of a session: the instance's own
    prices shifted by k hours (one row per stage of the horizon)."""
    from synth.problems import day_night_price
    N = P["tree"]["horizon"]
    base = P["alpha2"] / np.maximum(day_night_price(N, 0)[:, None], 1e-300)
    return day_night_price(N, t0=k)[:, None] * base


def _session_request(P, k, x, q):
    """MPC step k of a session: measured state x, previous input q, forecast and prices
    shifted by k hours from the instance's own start hour."""
    import synth
    N = P["tree"]["horizon"]
    dhat = synth.demand_forecast(P["net"], N, t0=k)
    return {"p": x, "q": q, "dhat": dhat, "alpha2": _session_prices(P, k)}


def closed_loop_kpis(u, x, alpha, u_before, x_s):
    """The closed-loop key performance indicators of Sec. V over H_s steps: u (H_s x n_u)
    the applied inputs, x (H_s x n_x) the states they led to, alpha (H_s x n_u) the prices
    alpha_1 + alpha_2,k of each step, u_before the input applied before the first step (for
    its Delta u), x_s the safety levels.
      KPI_E   = (1/H_s) sum_k (alpha_1 + alpha_2,k)' |u_k|         (average economic cost)
      KPI_dU  = (1/H_s) sum_k ||u_k - u_{k-1}||^2                  (smoothness of the inputs)
      KPI_S   = sum_k ||[x_s - x_k]_+||_1                          (water below the safety levels)
      KPI_R   = ||x_s||_1 / ((1/H_s) sum_k ||x_k||_1) x 100 %      (safety level against the mean storage)"""
    u, x, alpha = (np.asarray(a, float) for a in (u, x, alpha))
    H = u.shape[0]
    du = np.diff(np.vstack([np.asarray(u_before, float)[None, :], u]), axis=0)
    return {"KPI_E": float(np.sum(alpha * np.abs(u)) / H),
            "KPI_dU": float(np.sum(du ** 2) / H),
            "KPI_S": float(np.sum(np.maximum(np.asarray(x_s, float)[None, :] - x, 0.0))),
            "KPI_R_pct": float(np.abs(x_s).sum() / (np.abs(x).sum(axis=1).mean()) * 100.0),
            "steps": int(H)}


def _record_step(s_, k, u0):
    """Applies a session's step-k input to its plant and keeps the closed-loop trajectory
    (input, resulting state, prices of the step) for the KPIs."""
    P = s_["P"]
    s_["x"] = _plant_step(P, s_["x"], u0, k, s_["rng"])
    s_["traj"].append((u0.copy(), s_["x"].copy(), P["cost"]["alpha1"] + _session_prices(P, k)[0]))


def _plant_step(P, x, u0, k, rng):
    """Tank mass balance x+ = x + B u_0 + G_d d with the realised demand (forecast plus
    10 % noise), clipped to the tank capacities."""
    import synth
    net = P["net"]
    d = synth.demand_forecast(net, 1, t0=k)[0]
    d = d * (1 + 0.1 * rng.standard_normal(d.shape))
    return np.clip(x + net["B"] @ u0 + net["Gd"] @ d, 0.0, net["cap"])


def _serve_window(smpc, server, sess, rate, seconds, drain, args, rng):
    """Poisson arrivals at `rate` requests/s for `seconds`, then a drain; returns the
    window's completed solves and their latencies."""
    lat, queue_ms, run_ms, its, rho = [], [], [], [], []
    offered = 0
    t0 = time.perf_counter()
    next_arrival = t0 + rng.exponential(1.0 / rate)
    arrivals_end = t0 + seconds

    def poll_all():
        for s_ in sess:
            while s_["pending"]:
                tk, ts, k = s_["pending"][0]
                u0 = np.zeros(s_["P"]["net"]["n_u"])
                r = smpc.smpc_poll(server, tk, u0_host=u0)
                if r is None:
                    break
                s_["pending"].pop(0)
                lat.append(1000.0 * (time.perf_counter() - ts))
                queue_ms.append(r["queue_ms"])
                run_ms.append(r["run_ms"])
                its.append(r["iterations"])
                rho.append(r["rho_rel"])
                _record_step(s_, k, u0)
                s_["q"] = u0

    while True:
        now = time.perf_counter()
        while now < arrivals_end and next_arrival <= now:
            s_ = sess[int(rng.integers(len(sess)))]
            req = _session_request(s_["P"], s_["k"], s_["x"], s_["q"])
            tk = smpc.smpc_submit(server, s_["fac"], req["p"], req["q"], req["dhat"], req["alpha2"], eps=s_["P"]["eps"],
                                  max_iters=args.serve_max_iters, tol=args.tol, warm_start=int(s_["k"] > 0),
                                  check_every=64)
            s_["pending"].append((tk, time.perf_counter(), s_["k"]))
            s_["k"] += 1
            offered += 1
            next_arrival += rng.exponential(1.0 / rate)
        poll_all()
        outstanding = sum(len(s_["pending"]) for s_ in sess)
        if now >= arrivals_end and (outstanding == 0 or now > arrivals_end + drain):
            break
        time.sleep(0.0002)
    elapsed = time.perf_counter() - t0
    done = len(lat)
    rho = np.asarray(rho)
    return {"offered_rate": rate, "offered": offered, "completed": done, "seconds": elapsed,
            "solves_per_s": done / elapsed, "unfinished": sum(len(s_["pending"]) for s_ in sess),
            "reached_tol": int((rho <= args.tol).sum()), "max_rho_rel": float(rho.max()) if done else None,
            "p50_ms": float(np.percentile(lat, 50)) if lat else None,
            "p99_ms": float(np.percentile(lat, 99)) if lat else None,
            "queue_p50_ms": float(np.percentile(queue_ms, 50)) if lat else None,
            "run_p50_ms": float(np.percentile(run_ms, 50)) if lat else None,
            "iterations_mean": float(np.mean(its)) if its else None}


def serve_kpis(sess):
    """Each session's closed-loop KPIs over the steps it completed (the requests are solved
    in order per session), and their mean and range over the sessions."""
    per = []
    for s_ in sess:
        if not s_["traj"]:
            continue
        u, x, a = (np.array([t[i] for t in s_["traj"]]) for i in range(3))
        per.append(closed_loop_kpis(u, x, a, s_["q_start"], s_["P"]["cost"]["x_s"]))
    if not per:
        return None
    out = {"sessions": len(per), "steps_per_session_mean": float(np.mean([p["steps"] for p in per])),
           "definitions": "Sec. V: KPI_E average economic cost (alpha_1 + alpha_2,k)'|u_k|; KPI_dU average "
                          "||u_k - u_(k-1)||^2; KPI_S total ||[x_s - x_k]_+||_1; KPI_R ||x_s||_1 over the mean "
                          "||x_k||_1, in %; per session over its completed steps, then over the sessions"}
    for key in ("KPI_E", "KPI_dU", "KPI_S", "KPI_R_pct"):
        v = np.array([p[key] for p in per])
        out[key] = {"mean": float(v.mean()), "min": float(v.min()), "max": float(v.max())}
    return out


def run_serve(args):
    """Closed-loop serving (Alg. 2 for 64 controllers): Poisson arrivals at a sweep of
    offered rates, each request a warm-started solve to rho_rel <= tol (no effective
    iteration cap), continuous batching through the server's slots.  Reports every
    rate's throughput and latency, and the highest rate the GPU sustained (completed
    >= 95 % of offered, nothing left over, median queueing no longer than the median
    solve); the FP64 per-request solve of the same closed loop beside it."""
    import torch

    import paper_1604_01074_gb300 as smpc
    import synth
    torch.cuda.set_device(0)
    insts = synth.batch_instances(0)
    log("serve: building", len(insts), "factors")
    sess = []
    for i, P in enumerate(insts):
        t = P["tree"]
        tree = smpc.smpc_tree_create(t["parent"], t["prob"])
        prec = 1 if i % 2 == 0 else 2  # float32 and bfloat16 packs, mixed
        fac = smpc.smpc_factor(tree, P["net"], P["cost"], precision=prec, precondition=1, shared_packs=1)
        sess.append({"P": P, "tree": tree, "fac": fac, "prec": prec, "x": P["p"].copy(), "q": P["q"].copy(),
                     "k": 0, "pending": [], "rng": np.random.default_rng(100 + i), "traj": [],
                     "q_start": P["q"].copy()})
    total_bytes = sum(smpc.smpc_factor_device_bytes(s_["fac"]) for s_ in sess)
    log("serve: factors ready,", total_bytes / 1e9, "GB")
    budget = int(args.serve_budget_gb * 1e9)
    server = smpc.smpc_server_create(budget, args.serve_slots)
    rng = np.random.default_rng(0)
    # every session's first (cold) step, untimed: the closed loops start warm
    for s_ in sess:
        req = _session_request(s_["P"], 0, s_["x"], s_["q"])
        tk = smpc.smpc_submit(server, s_["fac"], req["p"], req["q"], req["dhat"], req["alpha2"], eps=s_["P"]["eps"],
                              max_iters=args.serve_max_iters, tol=args.tol, check_every=64)
        s_["pending"].append((tk, time.perf_counter(), 0))
        s_["k"] = 1
    t_cold = time.perf_counter()
    n_cold = 0
    while any(s_["pending"] for s_ in sess):
        for s_ in sess:
            if s_["pending"]:
                tk, _, k = s_["pending"][0]
                u0 = np.zeros(s_["P"]["net"]["n_u"])
                r = smpc.smpc_poll(server, tk, u0_host=u0)
                if r is not None:
                    s_["pending"].pop(0)
                    _record_step(s_, k, u0)
                    s_["q"] = u0
                    n_cold += 1
                    log("serve: cold step", n_cold, "of", len(sess), "session", sess.index(s_), "nodes",
                        len(s_["P"]["tree"]["parent"]), "prec", s_["prec"], "iterations", r["iterations"],
                        "rho_rel", round(r["rho_rel"], 6), "run_ms", round(r["run_ms"], 1), "at",
                        round(time.perf_counter() - t_cold, 2))
        time.sleep(0.001)
    log("serve: cold steps done in", time.perf_counter() - t_cold, "s")
    windows = []
    for rate in args.serve_rates:
        w = _serve_window(smpc, server, sess, rate, args.serve_seconds, args.serve_drain, args, rng)
        windows.append(w)
        log("serve window", w)
        if w["unfinished"] > 0 or w["completed"] < 0.95 * w["offered"]:
            break  # saturated: higher rates only grow the queue
    smpc.smpc_server_destroy(server)
    # sustained: every request served within the window and queueing below the solve time itself
    sustained = [w for w in windows if w["unfinished"] == 0 and w["completed"] >= 0.95 * w["offered"]
                 and (w["queue_p50_ms"] or 0.0) <= (w["run_p50_ms"] or 0.0)]
    best = max(sustained, key=lambda w: w["offered_rate"]) if sustained else windows[0]
    result = {
        "metric": "SMPC serving: solves/s and p50/p99 latency (ms), closed loop, tol 1e-3", "impl": "ours-serve",
        "value": best["solves_per_s"], "unit": "solves/s", "sustained_rate": best["offered_rate"],
        "p50_ms": best["p50_ms"], "p99_ms": best["p99_ms"], "reached_tol_fraction":
            best["reached_tol"] / max(1, best["completed"]), "windows": windows,
        "config": {"workload": SERVE_WORKLOAD, "slots": args.serve_slots, "hbm_budget_bytes": budget,
                   "factor_bytes_total": total_bytes, "precision": "fp32 and bf16 shared packs, alternating by session",
                   "max_iters": args.serve_max_iters, "tol": args.tol, "warm_start": "each session's previous step",
                   "launch": "plain launches, 64-iteration chunks between stop checks", "rates": args.serve_rates,
                   "window_s": args.serve_seconds}}
    result["closed_loop_kpis"] = serve_kpis(sess)
    # baseline: the plain per-request FP64 solve (one pack per node), one at a time, on a
    # sample of sessions continuing their closed loops (warm-started steps, same tol)
    base, base_it = [], []
    for s_ in sess[: args.serve_baseline]:
        P = s_["P"]
        f64 = smpc.smpc_factor(s_["tree"], P["net"], P["cost"], precision=0, precondition=1)
        x, q = P["p"].copy(), P["q"].copy()
        for k in range(3):
            req = _session_request(P, k, x, q)
            u0 = np.zeros(P["net"]["n_u"])
            torch.cuda.synchronize()
            ts = time.perf_counter()
            info = smpc.smpc_solve(f64, req["p"], req["q"], req["dhat"], req["alpha2"], eps=P["eps"],
                                   max_iters=args.serve_max_iters, tol=args.tol, warm_start=int(k > 0), sync=1,
                                   u0_host=u0)
            if k > 0:
                base.append(1000.0 * (time.perf_counter() - ts))
                base_it.append(info["iterations"])
            x = _plant_step(P, x, u0, k, s_["rng"])
            q = u0
        smpc.smpc_factor_destroy(f64)
    if base:
        result["fp64_per_request"] = {"mean_ms": float(np.mean(base)), "p50_ms": float(np.percentile(base, 50)),
                                      "p99_ms": float(np.percentile(base, 99)),
                                      "solves_per_s": 1000.0 / float(np.mean(base)),
                                      "iterations_mean": float(np.mean(base_it)),
                                      "sample": f"{len(base)} warm-started steps of {args.serve_baseline} sessions, "
                                                "same tol"}
    for s_ in sess:
        smpc.smpc_factor_destroy(s_["fac"])
        smpc.smpc_tree_destroy(s_["tree"])
    return result


# --------------------------------------------------------------------- batched (forests)
def run_batched(args):
    """The 64 instances as four forests (one per network: the instances sharing a network
    are one factor whose mat-vecs run as GEMMs over one shared pack), the four forests in
    one batch (smpc_batch_solve: one CUDA graph per chunk of iterations, one branch per
    forest).  Every tree stops at its own first iterate with rho_rel <= tol.  Baseline: the
    plain FP64 single-tree solve (one pack per node) of every instance, one at a time."""
    import torch

    import paper_1604_01074_gb300 as smpc
    import synth
    torch.cuda.set_device(0)
    insts = synth.batch_instances(0)
    groups = [[P for P in insts if P["network"] == k] for k in range(4)]
    prec = {"fp64": 0, "fp32": 1, "bf16": 2}[args.batched_precision]
    forests, facs, trees = [], [], []
    t0 = time.perf_counter()
    for grp in groups:
        F = synth.forest(grp)
        t = F["tree"]
        tree = smpc.smpc_tree_create(t["parent"], t["prob"])
        fac = smpc.smpc_factor(tree, F["net"], F["cost"], precision=prec, precondition=1, shared_packs=1)
        forests.append(F)
        facs.append(fac)
        trees.append(tree)
    setup_s = time.perf_counter() - t0
    log("batched: factors ready in", setup_s, "s; schedules", [smpc.smpc_factor_schedule(f)[0] for f in facs])
    batch = smpc.smpc_batch_create(facs)
    stream = torch.cuda.current_stream()
    runs = []
    for rep_ in range(args.batched_reps + 1):  # the first run captures the graphs (untimed)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = smpc.smpc_batch_solve(batch, forests, max_iters=args.max_iters, tol=args.tol, check_every=64,
                                    use_graph=1, stream=stream)
        e1.record(stream)
        e1.synchronize()
        per_tree = [smpc.smpc_solve_trees(f, len(g)) for f, g in zip(facs, groups)]
        runs.append((e0.elapsed_time(e1) / 1000.0, res, per_tree))
        log("batched rep", rep_, runs[-1][0], [r["iterations"] for r in res])
    smpc.smpc_batch_destroy(batch)
    timed = runs[1:] if len(runs) > 1 else runs
    wall, res, per_tree = min(timed, key=lambda x: x[0])
    n_inst = sum(len(g) for g in groups)
    rr_all = np.concatenate([rr for _, rr in per_tree])
    it_all = np.concatenate([it for it, _ in per_tree])
    out = {"metric": "SMPC solves/sec to 1e-3 primal-dual residual, batched (64 uneven trees on 4 networks)",
           "impl": "ours-batched", "value": n_inst / wall, "unit": "solves/s", "wall_s": wall,
           "reached_tol": int((rr_all <= args.tol).sum()), "trees": n_inst, "max_tree_rho_rel": float(rr_all.max()),
           "tree_iterations": {"min": int(it_all.min()), "mean": float(it_all.mean()), "max": int(it_all.max())},
           "forests": [{"trees": len(g), "nodes": int(len(F["tree"]["parent"])), "iterations": r["iterations"],
                        "tree_rho_rel_max": float(rr.max()), "tree_iterations": it.tolist()}
                       for g, F, r, (it, rr) in zip(groups, forests, res, per_tree)],
           "config": {"workload": "64 instances, 4 networks (n_x, n_u) in {(20,40),(35,65),(50,90),(63,114)}, "
                                  "N in {12,18,24}, 10-500 scenarios, 249,644 nodes",
                      "precision": args.batched_precision, "packs": "shared (one per forest)",
                      "launch": "one smpc_batch_solve: each 64-iteration chunk of all four forests is one CUDA "
                                "graph with one branch per forest", "tol": args.tol,
                      "criterion": "every tree stops at its own first iterate with rho_rel <= tol (its own residual "
                                   "and scale)", "factor_setup_s": setup_s, "timing": "CUDA events, best of "
                                   f"{len(timed)} runs after a capture run"}}
    for f_, t_ in zip(facs, trees):
        smpc.smpc_factor_destroy(f_)
        smpc.smpc_tree_destroy(t_)
    # the plain FP64 single-tree solve of every instance (one pack per node), one at a time
    base, base_it = 0.0, []
    sample = insts[: args.batched_baseline] if args.batched_baseline > 0 else insts
    for P in sample:
        t = P["tree"]
        tree = smpc.smpc_tree_create(t["parent"], t["prob"])
        fac = smpc.smpc_factor(tree, P["net"], P["cost"], precision=0, precondition=1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = smpc.smpc_solve(fac, P["p"], P["q"], P["dhat"], P["alpha2"], eps=P["eps"], max_iters=args.max_iters,
                               tol=args.tol, sync=1, stream=stream)
        e1.record(stream)
        e1.synchronize()
        base += e0.elapsed_time(e1) / 1000.0
        base_it.append(info["iterations"])
        smpc.smpc_factor_destroy(fac)
        smpc.smpc_tree_destroy(tree)
    out["fp64_single_tree"] = {"solves_per_s": len(sample) / base, "total_s": base, "instances": len(sample),
                               "iterations_mean": float(np.mean(base_it)),
                               "note": "every instance solved alone to the same tol, FP64 per-node packs"}
    out["speedup_vs_fp64_single_tree"] = out["value"] / out["fp64_single_tree"]["solves_per_s"]
    return out


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle as it stands, on the host cores, for the same
    workload and metric.  Each step is a bounded sample of the workload (about 6 s of
    APG iterations on one MPC step's inputs); ms_per_step is that sample's measured
    time, and value scales the measured iteration rate to whole solves by the oracle's
    own iteration count to rho_rel <= 1e-3."""
    if rank != 0:
        return None
    stored, meta = oracle_iters_to_tol(args.config)
    iters_to_tol = stored
    if iters_to_tol is None:
        return {"impl": "reference", "unavailable": "no stored oracle iteration count for this workload"}
    probe = run_oracle_sample(args.config, 3)
    per = max(3, min(400, int(6000.0 / max(probe["ms_per_iter"], 1e-3))))
    for k in range(args.warmup):
        run_oracle_sample(args.config, max(2, per // 10), step=k)
    samples = [run_oracle_sample(args.config, per, step=args.warmup + k) for k in range(args.steps)]
    ms_iter = statistics.mean(s_["ms_per_iter"] for s_ in samples)
    ms_step = statistics.mean(s_["seconds"] * 1000.0 for s_ in samples)
    value = 1000.0 / (ms_iter * iters_to_tol)
    sample = (f"{per} FP64 APG iterations per step ({per / iters_to_tol:.4f} of a solve), iteration rate scaled "
              f"to {iters_to_tol} iterations per solve (the oracle's own count to 1e-3)")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.config], "tol": args.tol,
                       "implementation": "FP64 CPU oracle (numpy), one host core",
                       "step": f"a bounded sample: {per} APG iterations of one MPC step's inputs"},
            "apg_iters_per_s": 1000.0 / ms_iter, "solve_fraction_per_step": per / iters_to_tol,
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": sample,
                             "host_cores": os.cpu_count()},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def spawn_ranks(n):
    """--gpus N outside torchrun: run N ranks of this script through torch.distributed.run
    (one process per GPU, rendezvous on 127.0.0.1) and return its exit code."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr", "127.0.0.1", "--master-port", str(29500 + os.getpid() % 1000),
           os.path.abspath(__file__), *sys.argv[1:]]
    return subprocess.call(cmd, cwd=ROOT)


def _jsonable(o):
    if hasattr(o, "item"):
        return o.item()
    if isinstance(o, (set, tuple)):
        return list(o)
    return str(o)


def log(*a):
    print("[bench]", *a, file=sys.stderr, flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "fp32", "bf16"], default="fp32")
    ap.add_argument("--config", choices=["barcelona", "tiny", "large"], default="large")
    ap.add_argument("--tol", type=float, default=1e-3)
    ap.add_argument("--schedule", type=int, choices=[0, 1, 2, 3, 4], default=0,
                    help="iteration schedule: 0 = the factor times both and keeps the faster")
    ap.add_argument("--max-iters", type=int, default=100000)
    ap.add_argument("--no-graph", action="store_true", help="plain launches instead of CUDA-graph chunks")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3, help="solves timed end to end (at most --steps)")
    ap.add_argument("--leg-solves", type=int, default=3, help="legs: solves timed per leg")
    ap.add_argument("--no-other-precisions", dest="other_legs", action="store_false")
    ap.add_argument("--oracle-sample", type=int, default=0)
    ap.add_argument("--oracle-step", type=int, default=0)
    ap.add_argument("--oracle-start", type=float, default=0.0)
    ap.add_argument("--serve", action="store_true", help="closed-loop serving workload (its own JSON line)")
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[2.0, 4.0, 8.0, 16.0, 32.0, 64.0, 200.0])
    ap.add_argument("--serve-seconds", type=float, default=20.0)
    ap.add_argument("--serve-drain", type=float, default=30.0)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-budget-gb", type=float, default=64.0)
    ap.add_argument("--serve-max-iters", type=int, default=100000)
    ap.add_argument("--serve-baseline", type=int, default=6)
    ap.add_argument("--batched", action="store_true", help="the 64-instance batched workload (its own JSON line)")
    ap.add_argument("--batched-precision", choices=["fp64", "fp32", "bf16"], default="bf16")
    ap.add_argument("--batched-reps", type=int, default=2)
    ap.add_argument("--batched-baseline", type=int, default=0,
                    help="instances in the FP64 single-tree baseline (0: all 64)")
    ap.add_argument("--shared-packs", action="store_true", help="--profile-solve: one shared pack per factor")
    ap.add_argument("--profile-solve", type=int, default=0,
                    help="factor, a warm-up solve, then one solve of this many iterations (tol 0) inside a "
                         "CUDA profiler range, and exit: the case ncu captures (--profile-from-start off)")
    args = ap.parse_args()
    if args.oracle_sample:
        oracle_sample(args.config, args.oracle_sample, args.oracle_step, args.oracle_start)
        return
    if args.profile_solve:
        profile_solve(args)
        return
    if args.serve:
        print(json.dumps(run_serve(args), default=_jsonable))
        return
    if args.batched:
        print(json.dumps(run_batched(args), default=_jsonable))
        return
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(spawn_ranks(args.gpus))
    rank, world, local_rank = dist_env()
    if args.impl == "reference":
        res = run_reference(args, rank, world)
    else:
        res = run_ours(args, rank, world, local_rank)
    if rank == 0 and res is not None:
        print(json.dumps(res, default=_jsonable))


if __name__ == "__main__":
    main()
