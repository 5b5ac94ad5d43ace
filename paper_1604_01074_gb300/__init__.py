"""Python binding of libsmpc.so: the C ABI declared in include/smpc.h, same names.

Argument marshalling only: every step of the solver runs in the library's CUDA
kernels.  PyTorch tensors serve as device buffers (``data_ptr()``) and their
stream handles are passed through.  The library must have been built
(``__graft_entry__.build()``); there is no fallback of any kind.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsmpc.so")

SMPC_OK, SMPC_EINVAL, SMPC_ENOMEM, SMPC_ECUDA, SMPC_EBUSY, SMPC_ETIMEOUT, SMPC_EDIVERGED, SMPC_ENOTSUP = range(8)
SMPC_MAX_ITERS = 1 << 26  # include/smpc.h: the largest max_iters a solve accepts
SMPC_FP64, SMPC_FP32, SMPC_BF16 = 0, 1, 2

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)


class smpc_network(ctypes.Structure):
    _fields_ = [("n_x", ctypes.c_int32), ("n_u", ctypes.c_int32), ("n_d", ctypes.c_int32), ("n_e", ctypes.c_int32),
                ("A", _dp), ("B", _dp), ("Gd", _dp), ("E", _dp), ("Ed", _dp)]


class smpc_cost(ctypes.Structure):
    _fields_ = [("W_alpha", ctypes.c_double), ("alpha1", _dp), ("W_u", _dp), ("W_x", ctypes.c_double),
                ("gamma_d", ctypes.c_double), ("x_min", _dp), ("x_max", _dp), ("x_s", _dp), ("u_min", _dp),
                ("u_max", _dp), ("safety_unweighted", ctypes.c_int32)]


class smpc_factor_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("precondition", ctypes.c_int32), ("lambda_", ctypes.c_double),
                ("power_iters", ctypes.c_int32), ("lambda_margin", ctypes.c_double),
                ("step_s", _dp), ("step_z", _dp), ("step_p", _dp), ("shared_packs", ctypes.c_int32),
                ("schedule", ctypes.c_int32), ("tc_width", ctypes.c_int32)]


class smpc_step_data(ctypes.Structure):
    _fields_ = [("p", _dp), ("q", _dp), ("dhat", _dp), ("eps", _dp), ("alpha2", _dp)]


class smpc_solve_opts(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_int32), ("tol", ctypes.c_double), ("warm_start", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("sync", ctypes.c_int32), ("polish_iters", ctypes.c_int32),
                ("anchor_every", ctypes.c_int32), ("use_graph", ctypes.c_int32), ("ergodic", ctypes.c_int32)]


class smpc_result(ctypes.Structure):
    _fields_ = [("u", ctypes.c_void_p), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("u0_host", _dp),
                ("history_host", _dp), ("iterations", ctypes.c_int32), ("rho", ctypes.c_double),
                ("rho_rel", ctypes.c_double), ("launches", ctypes.c_int32), ("queue_ms", ctypes.c_double),
                ("run_ms", ctypes.c_double), ("ubar", ctypes.c_void_p), ("xbar", ctypes.c_void_p)]


class smpc_tree_info(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int32), ("horizon", ctypes.c_int32), ("n_leaves", ctypes.c_int32),
                ("n_chains", ctypes.c_int32), ("n_top", ctypes.c_int32), ("max_chain_len", ctypes.c_int32), ("n_trees", ctypes.c_int32)]


# symbol -> (restype, argtypes); every entry point declared in include/smpc.h
SIGNATURES = {
    "smpc_tree_create": (ctypes.c_int, [ctypes.c_int32, _ip, _dp, ctypes.POINTER(ctypes.c_void_p)]),
    "smpc_tree_info_get": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(smpc_tree_info)]),
    "smpc_tree_destroy": (None, [ctypes.c_void_p]),
    "smpc_factor": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(smpc_network), ctypes.POINTER(smpc_cost),
                                   ctypes.POINTER(smpc_factor_opts), ctypes.POINTER(ctypes.c_void_p)]),
    "smpc_factor_destroy": (None, [ctypes.c_void_p]),
    "smpc_factor_steps": (ctypes.c_int, [ctypes.c_void_p, _dp, _dp, _dp, _dp]),
    "smpc_factor_schedule": (ctypes.c_int, [ctypes.c_void_p, _dp]),
    "smpc_factor_device_bytes": (ctypes.c_size_t, [ctypes.c_void_p]),
    "smpc_server_create": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)]),
    "smpc_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(smpc_step_data),
                                   ctypes.POINTER(smpc_solve_opts), ctypes.POINTER(ctypes.c_uint64)]),
    "smpc_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(smpc_result),
                                 ctypes.POINTER(ctypes.c_int32)]),
    "smpc_server_destroy": (None, [ctypes.c_void_p]),
    "smpc_profile_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(smpc_step_data), ctypes.c_int32, _dp,
                                          ctypes.c_int32]),
    "smpc_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(smpc_step_data), ctypes.POINTER(smpc_solve_opts),
                                  ctypes.POINTER(smpc_result), ctypes.c_void_p]),
    "smpc_solve_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(smpc_result)]),
    "smpc_solve_static": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(smpc_step_data),
                                         ctypes.POINTER(smpc_solve_opts), ctypes.POINTER(smpc_result), ctypes.c_void_p]),
    "smpc_fma_peak": (ctypes.c_int, [ctypes.c_int32, _dp]),
    "smpc_solve_trees": (ctypes.c_int, [ctypes.c_void_p, _ip, _dp]),
    "smpc_factor_tc_width": (ctypes.c_int, [ctypes.c_void_p, _dp]),
    "smpc_batch_create": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p),
                                         ctypes.POINTER(ctypes.c_void_p)]),
    "smpc_batch_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(smpc_step_data),
                                        ctypes.POINTER(smpc_solve_opts), ctypes.POINTER(smpc_result), ctypes.c_void_p]),
    "smpc_batch_destroy": (None, [ctypes.c_void_p]),
    "smpc_shard_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_void_p)]),
    "smpc_shard_info": (ctypes.c_int, [ctypes.c_void_p, _ip, _ip, _ip]),
    "smpc_shard_nodes": (ctypes.c_int, [ctypes.c_void_p, _ip]),
    "smpc_shard_begin": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(smpc_step_data),
                                        ctypes.POINTER(smpc_solve_opts), ctypes.c_void_p, ctypes.c_void_p]),
    "smpc_shard_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]),
    "smpc_shard_flags": (ctypes.c_int, [ctypes.c_void_p, _ip, _ip]),
    "smpc_shard_finish": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(smpc_result)]),
    "smpc_shard_destroy": (None, [ctypes.c_void_p]),
    "smpc_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "smpc_last_error": (ctypes.c_char_p, []),
    "smpc_version": (ctypes.c_int, []),
}

_lib = None


def lib():
    """Load libsmpc.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing; build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class SmpcError(RuntimeError):
    def __init__(self, code, where):
        L = lib()
        super().__init__(f"{where}: {L.smpc_status_string(code).decode()} ({code}): {L.smpc_last_error().decode()}")
        self.code = code


def _check(code, where):
    if code != SMPC_OK:
        raise SmpcError(code, where)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_dp)


class _Keep:
    """Holds numpy arrays alive while a call uses their pointers."""

    def __init__(self):
        self.arrays = []

    def __call__(self, a):
        if a is None:
            return None
        a = _f64(a)
        self.arrays.append(a)
        return _ptr(a)


# --------------------------------------------------------------------- the calls
def smpc_tree_create(parent, prob=None):
    parent = np.ascontiguousarray(np.asarray(parent, dtype=np.int32))
    prob_a = None if prob is None else _f64(prob)
    h = ctypes.c_void_p()
    _check(lib().smpc_tree_create(len(parent), parent.ctypes.data_as(_ip), _ptr(prob_a), ctypes.byref(h)),
           "smpc_tree_create")
    return h


def smpc_tree_info_get(tree):
    info = smpc_tree_info()
    _check(lib().smpc_tree_info_get(tree, ctypes.byref(info)), "smpc_tree_info_get")
    return {k: getattr(info, k) for k, _ in smpc_tree_info._fields_}


def smpc_tree_destroy(tree):
    lib().smpc_tree_destroy(tree)


def smpc_factor(tree, net, cost, precision=SMPC_FP64, precondition=1, lam=0.0, power_iters=0, lambda_margin=0.0,
                steps=None, safety_unweighted=0, schedule=0, shared_packs=0, tc_width=0):
    """net / cost: dicts with the fields of smpc_network / smpc_cost (numpy arrays).
    steps: optional dict {'s': (n,), 'z': (n,), 'p': (n, n_u)} of explicit per-entry steps.
    schedule: 0 = time the iteration schedules and keep the fastest, 1 = chain, 2 = node, 3 = hybrid,
    4 = fused chain pass."""
    k = _Keep()
    A = net.get("A")
    n_x, n_u = net["B"].shape
    n_d = net["Gd"].shape[1]
    n_e = net["E"].shape[0] if net.get("E") is not None else 0
    N = smpc_network(n_x, n_u, n_d, n_e, k(A), k(net["B"]), k(net["Gd"]),
                     k(net["E"]) if n_e else None, k(net["Ed"]) if n_e else None)
    C = smpc_cost(float(cost["W_alpha"]), k(cost["alpha1"]), k(cost["W_u"]), float(cost["W_x"]), float(cost["gamma_d"]),
                  k(cost["x_min"]), k(cost["x_max"]), k(cost["x_s"]), k(cost["u_min"]), k(cost["u_max"]),
                  int(safety_unweighted))
    O = smpc_factor_opts(int(precision), int(precondition), float(lam), int(power_iters), float(lambda_margin),
                         None, None, None, int(shared_packs), int(schedule), int(tc_width))
    if steps is not None:
        O.step_s, O.step_z, O.step_p = k(steps["s"]), k(steps["z"]), k(steps["p"])
    h = ctypes.c_void_p()
    _check(lib().smpc_factor(tree, ctypes.byref(N), ctypes.byref(C), ctypes.byref(O), ctypes.byref(h)), "smpc_factor")
    return h


def smpc_factor_destroy(fac):
    lib().smpc_factor_destroy(fac)


def smpc_factor_schedule(fac):
    """(schedule in use, {schedule: ms per iteration} as timed by the factor)."""
    ms = (ctypes.c_double * 4)()
    s = lib().smpc_factor_schedule(fac, ms)
    if s < 0:
        raise SmpcError(-s, smpc_last_error())
    return s, {1: ms[0], 2: ms[1], 3: ms[2], 4: ms[3]}


def smpc_factor_tc_width(fac):
    """(nodes per tensor-core GEMM or 0, {16: ms, 32: ms, 64: ms} as timed by the factor)."""
    ms = (ctypes.c_double * 3)()
    w = lib().smpc_factor_tc_width(fac, ms)
    if w < 0:
        raise SmpcError(-w, smpc_last_error())
    return w, {16: ms[0], 32: ms[1], 64: ms[2]}


def smpc_factor_steps(fac, n, n_u):
    lam = ctypes.c_double()
    s, z, p = np.zeros(n), np.zeros(n), np.zeros((n, n_u))
    _check(lib().smpc_factor_steps(fac, ctypes.byref(lam), _ptr(s), _ptr(z), _ptr(p)), "smpc_factor_steps")
    return lam.value, {"s": s, "z": z, "p": p}


def smpc_solve(fac, p, q, dhat, alpha2, eps=None, max_iters=500, tol=0.0, warm_start=0, check_every=0, sync=1,
               u=None, x=None, y=None, u0_host=None, history_host=None, stream=None, polish_iters=0,
               anchor_every=0, use_graph=0, ergodic=0, ubar=None, xbar=None, _entry="smpc_solve"):
    """u, x, y: optional torch device tensors (or raw device pointers) receiving the outputs.
    u0_host / history_host: optional numpy float64 arrays filled when sync=1.  use_graph=1
    enqueues each chunk of iterations as a CUDA graph, captured once per chunk and
    settings and replayed by later solves of the factor.  ergodic=1 keeps the ergodic
    primal average, copied to the device tensors ubar and xbar."""
    k = _Keep()

    def arg(a):  # host array, or an int device address of float64 data
        if isinstance(a, int):
            return ctypes.cast(ctypes.c_void_p(a), _dp)
        return k(a)

    D = smpc_step_data(arg(p), arg(q), arg(dhat), arg(eps), arg(alpha2))
    O = smpc_solve_opts(int(max_iters), float(tol), int(warm_start), int(check_every), int(sync), int(polish_iters),
                        int(anchor_every), int(use_graph), int(ergodic))

    def dptr(t):
        if t is None:
            return None
        return t if isinstance(t, int) else t.data_ptr()

    R = smpc_result(dptr(u), dptr(x), dptr(y),
                    None if u0_host is None else u0_host.ctypes.data_as(_dp),
                    None if history_host is None else history_host.ctypes.data_as(_dp), -1, 0.0, 0.0, 0, 0.0, 0.0,
                    dptr(ubar), dptr(xbar))
    if stream is None:
        s = None
    elif isinstance(stream, int):
        s = stream
    else:
        s = stream.cuda_stream
    _check(getattr(lib(), _entry)(fac, ctypes.byref(D), ctypes.byref(O), ctypes.byref(R), s), _entry)
    return {"iterations": R.iterations, "rho": R.rho, "rho_rel": R.rho_rel, "launches": R.launches}


def smpc_solve_static(fac, p, q, dhat, alpha2, eps=None, max_iters=500, tol=0.0, warm_start=0, check_every=0,
                      sync=1, u=None, x=None, y=None, u0_host=None, history_host=None, stream=None, polish_iters=0,
                      anchor_every=0, ergodic=0):
    """smpc_solve without memory allocation (scratch in the library's static device
    array); same arguments and results as smpc_solve (ergodic=1 is refused)."""
    return smpc_solve(fac, p, q, dhat, alpha2, eps=eps, max_iters=max_iters, tol=tol, warm_start=warm_start,
                      check_every=check_every, sync=sync, u=u, x=x, y=y, u0_host=u0_host,
                      history_host=history_host, stream=stream, polish_iters=polish_iters,
                      anchor_every=anchor_every, ergodic=ergodic, _entry="smpc_solve_static")


def smpc_profile_solve(fac, p, q, dhat, alpha2, eps=None, iters=50):
    """Mean device ms of each kernel of an iteration over a cold-start solve of `iters`
    iterations (list: 1 entry for schedule 1, 5 for schedule 2)."""
    k = _Keep()

    def arg(a):
        if isinstance(a, int):
            return ctypes.cast(ctypes.c_void_p(a), _dp)
        return k(a)

    D = smpc_step_data(arg(p), arg(q), arg(dhat), arg(eps), arg(alpha2))
    out = (ctypes.c_double * 8)()
    n = lib().smpc_profile_solve(fac, ctypes.byref(D), int(iters), out, 8)
    if n < 0:
        raise SmpcError(-n, smpc_last_error())
    return [out[i] for i in range(n)]


def smpc_factor_device_bytes(fac):
    return int(lib().smpc_factor_device_bytes(fac))


def smpc_server_create(hbm_budget, max_slots):
    h = ctypes.c_void_p()
    _check(lib().smpc_server_create(int(hbm_budget), int(max_slots), ctypes.byref(h)), "smpc_server_create")
    return h


def smpc_server_destroy(server):
    lib().smpc_server_destroy(server)


def smpc_submit(server, fac, p, q, dhat, alpha2, eps=None, max_iters=500, tol=0.0, warm_start=0, check_every=0,
                polish_iters=0, anchor_every=0, use_graph=0, ergodic=0):
    """Queues one solve; returns its ticket.  Step data: numpy float64 arrays.  use_graph=1:
    the slot runs the solve's iteration chunks as CUDA graphs (captured once per factor,
    chunk and settings).  ergodic=1: keep the ergodic average (smpc_poll's ubar, xbar)."""
    k = _Keep()
    D = smpc_step_data(k(p), k(q), k(dhat), k(eps), k(alpha2))
    O = smpc_solve_opts(int(max_iters), float(tol), int(warm_start), int(check_every), 0, int(polish_iters),
                        int(anchor_every), int(use_graph), int(ergodic))
    t = ctypes.c_uint64()
    _check(lib().smpc_submit(server, fac, ctypes.byref(D), ctypes.byref(O), ctypes.byref(t)), "smpc_submit")
    return t.value


def smpc_poll(server, ticket, u=None, x=None, y=None, u0_host=None, history_host=None, ubar=None, xbar=None):
    """None while the ticket is queued or running; else the result dict (outputs copied)."""
    def dptr(t):
        return None if t is None else (t if isinstance(t, int) else t.data_ptr())

    R = smpc_result(dptr(u), dptr(x), dptr(y), None if u0_host is None else u0_host.ctypes.data_as(_dp),
                    None if history_host is None else history_host.ctypes.data_as(_dp), -1, 0.0, 0.0, 0, 0.0, 0.0,
                    dptr(ubar), dptr(xbar))
    done = ctypes.c_int32()
    _check(lib().smpc_poll(server, ctypes.c_uint64(ticket), ctypes.byref(R), ctypes.byref(done)), "smpc_poll")
    if not done.value:
        return None
    return {"iterations": R.iterations, "rho": R.rho, "rho_rel": R.rho_rel, "launches": R.launches,
            "queue_ms": R.queue_ms, "run_ms": R.run_ms}


def smpc_solve_info(fac, u0_host=None, history_host=None):
    """Completes an asynchronous solve and returns its host-side outputs."""
    R = smpc_result(None, None, None, None if u0_host is None else u0_host.ctypes.data_as(_dp),
                    None if history_host is None else history_host.ctypes.data_as(_dp), -1, 0.0, 0.0, 0)
    _check(lib().smpc_solve_info(fac, ctypes.byref(R)), "smpc_solve_info")
    return {"iterations": R.iterations, "rho": R.rho, "rho_rel": R.rho_rel, "launches": R.launches}


def smpc_batch_create(factors):
    arr = (ctypes.c_void_p * len(factors))(*[f.value if hasattr(f, "value") else f for f in factors])
    h = ctypes.c_void_p()
    _check(lib().smpc_batch_create(len(factors), arr, ctypes.byref(h)), "smpc_batch_create")
    return h


def smpc_batch_destroy(batch):
    lib().smpc_batch_destroy(batch)


def smpc_batch_solve(batch, steps, max_iters=500, tol=0.0, warm_start=0, check_every=0, sync=1, outputs=None,
                     u0_host=None, stream=None, polish_iters=0, anchor_every=0, use_graph=0, ergodic=0,
                     bar_outputs=None):
    """steps: one dict (p, q, dhat, alpha2, eps) per factor of the batch (numpy float64 or int
    device addresses).  outputs: optional list of (u, x, y) device tensors per factor;
    u0_host: optional list of numpy arrays (R * n_u per factor); with ergodic=1,
    bar_outputs: optional list of (ubar, xbar) device tensors per factor.  Returns one
    result dict per factor."""
    k = _Keep()

    def arg(a):
        if a is None:
            return None
        if isinstance(a, int):
            return ctypes.cast(ctypes.c_void_p(a), _dp)
        return k(a)

    n = len(steps)
    D = (smpc_step_data * n)(*[smpc_step_data(arg(d["p"]), arg(d["q"]), arg(d["dhat"]), arg(d.get("eps")),
                                              arg(d["alpha2"])) for d in steps])
    O = smpc_solve_opts(int(max_iters), float(tol), int(warm_start), int(check_every), int(sync), int(polish_iters),
                        int(anchor_every), int(use_graph), int(ergodic))

    def dptr(t):
        return None if t is None else (t if isinstance(t, int) else t.data_ptr())

    R = (smpc_result * n)()
    for i in range(n):
        u, x, y = outputs[i] if outputs else (None, None, None)
        ub, xb = bar_outputs[i] if bar_outputs else (None, None)
        R[i] = smpc_result(dptr(u), dptr(x), dptr(y), None if u0_host is None else u0_host[i].ctypes.data_as(_dp),
                           None, -1, 0.0, 0.0, 0, 0.0, 0.0, dptr(ub), dptr(xb))
    s = None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    _check(lib().smpc_batch_solve(batch, D, ctypes.byref(O), R, s), "smpc_batch_solve")
    return [{"iterations": r.iterations, "rho": r.rho, "rho_rel": r.rho_rel, "launches": r.launches} for r in R]


def smpc_shard_create(fac, chain_begin, chain_end):
    h = ctypes.c_void_p()
    _check(lib().smpc_shard_create(fac, int(chain_begin), int(chain_end), ctypes.byref(h)), "smpc_shard_create")
    return h


def smpc_shard_info(shard):
    """(n_cut, width, n_nodes): cut parents, entries per cut parent in the exchange, nodes updated."""
    a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib().smpc_shard_info(shard, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "smpc_shard_info")
    return a.value, b.value, c.value


def smpc_shard_nodes(shard):
    n = smpc_shard_info(shard)[2]
    out = np.zeros(n, dtype=np.int32)
    _check(lib().smpc_shard_nodes(shard, out.ctypes.data_as(_ip)), "smpc_shard_nodes")
    return out


def smpc_shard_begin(shard, p, q, dhat, alpha2, residuals, eps=None, max_iters=500, tol=0.0, warm_start=0,
                     stream=None):
    """residuals: an int device address of 3 (max_iters + 2) uint64 (the caller's buffer)."""
    k = _Keep()
    D = smpc_step_data(k(p), k(q), k(dhat), k(eps), k(alpha2))
    O = smpc_solve_opts(int(max_iters), float(tol), int(warm_start), 0, 0, 0, 0, 0)
    s = None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    _check(lib().smpc_shard_begin(shard, ctypes.byref(D), ctypes.byref(O), ctypes.c_void_p(residuals), s),
           "smpc_shard_begin")


def smpc_shard_step(shard, nu, phase, exchange=None):
    _check(lib().smpc_shard_step(shard, int(nu), int(phase), None if exchange is None else ctypes.c_void_p(exchange)),
           "smpc_shard_step")


def smpc_shard_flags(shard):
    d, e = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().smpc_shard_flags(shard, ctypes.byref(d), ctypes.byref(e)), "smpc_shard_flags")
    return d.value, e.value


def smpc_shard_finish(shard, launched, u=None, x=None, y=None):
    def dptr(t):
        return None if t is None else (t if isinstance(t, int) else t.data_ptr())
    R = smpc_result(dptr(u), dptr(x), dptr(y), None, None, -1, 0.0, 0.0, 0)
    _check(lib().smpc_shard_finish(shard, int(launched), ctypes.byref(R)), "smpc_shard_finish")
    return {"iterations": R.iterations, "rho": R.rho, "rho_rel": R.rho_rel}


def smpc_shard_destroy(shard):
    lib().smpc_shard_destroy(shard)


def smpc_solve_trees(fac, n_trees):
    """Per-tree (iterations, rho_rel) of the factor's last smpc_solve: numpy arrays of n_trees."""
    it = np.zeros(n_trees, dtype=np.int32)
    rr = np.zeros(n_trees)
    _check(lib().smpc_solve_trees(fac, it.ctypes.data_as(_ip), rr.ctypes.data_as(_dp)), "smpc_solve_trees")
    return it, rr


def smpc_fma_peak(precision):
    """Measured FMA throughput of the current GPU in TFLOP/s (SMPC_FP64 or SMPC_FP32)."""
    t = ctypes.c_double()
    _check(lib().smpc_fma_peak(int(precision), ctypes.byref(t)), "smpc_fma_peak")
    return t.value


def smpc_status_string(code):
    return lib().smpc_status_string(code).decode()


def smpc_last_error():
    return lib().smpc_last_error().decode()


def smpc_version():
    return lib().smpc_version()
