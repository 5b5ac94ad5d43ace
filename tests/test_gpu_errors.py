"""Error paths of the solve, reached without any GPU fault:

* SMPC_EDIVERGED: steps far above 1 / L make the APG iteration grow geometrically
  until the iterates overflow; device-resident step data holding a NaN (host data is
  refused before any device work) gives non-finite primal iterates at once (the prox
  maps a non-finite argument to 0, so the primal iterate is checked too).
* SMPC_ENOMEM: a factor whose per-node packs need more device memory than the GPU
  has (a 2-million-node tree with the 63-tank network in float64: about 430 GB);
  cudaMalloc refuses it and nothing is launched.
* SMPC_ETIMEOUT: a test-only bound of zero on node_mv's pack-pipeline waits (one
  non-blocking test; SMPC_PIPELINE_WAIT_NS, read when a factor is created) makes a wait
  whose copy has not landed yet give up;
  the CTA records the error, lets its copies in flight land under the normal 2 s
  bound and returns, and the other kernels of the solve see the error flag and exit.
* SMPC_EINVAL for an iteration cap above SMPC_MAX_ITERS (the per-iteration tables would
  be sized from it), from smpc_solve, smpc_submit and smpc_profile_solve (above 4096),
  before any allocation.
After each, the same process solves a fresh factor normally.
"""
import os

import numpy as np
import pytest

import oracle
import synth
from tests import harness as H

pytestmark = pytest.mark.gpu


def _healthy_after():
    P = synth.tiny(0)
    steps = H.tiny_steps(P)
    R = H.oracle_run(P, steps, 50)
    g = H.Gpu(P, steps=steps)
    try:
        info = g.solve(50)
        u, _, _ = g.arrays()
    finally:
        g.close()
    assert info["iterations"] == 50
    assert H.relerr(u, R.u) <= 1e-9


@pytest.mark.parametrize("precision", [0, 1])
def test_steps_far_above_one_over_l_report_ediverged(precision):
    import paper_1604_01074_gb300 as smpc
    P = synth.tiny(0)
    tree, fac, _ = H.oracle_build(P)
    st = oracle.jacobi_steps(fac, tree)
    big = {k: 1e3 * st[k] for k in ("s", "z", "p")}
    g = H.Gpu(P, steps=big, precision=precision)
    try:
        with pytest.raises(smpc.SmpcError) as ei:
            g.solve(4000)
        assert ei.value.code == smpc.SMPC_EDIVERGED, ei.value
    finally:
        g.close()
    _healthy_after()


def test_nan_in_device_step_data_reports_ediverged():
    import torch

    import paper_1604_01074_gb300 as smpc
    P = synth.tiny(0)
    g = H.Gpu(P, steps=H.tiny_steps(P))
    try:
        p = P["p"].copy()
        p[1] = np.nan
        with pytest.raises(smpc.SmpcError) as ei:  # host data: refused before any device work
            smpc.smpc_solve(g.fac, p, P["q"], P["dhat"], P["alpha2"], eps=P["eps"], max_iters=20, sync=1)
        assert ei.value.code == smpc.SMPC_EINVAL
        dev = {k: torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).cuda()
               for k, v in (("p", p), ("q", P["q"]), ("dhat", P["dhat"]), ("alpha2", P["alpha2"]), ("eps", P["eps"]))}
        with pytest.raises(smpc.SmpcError) as ei:
            smpc.smpc_solve(g.fac, dev["p"].data_ptr(), dev["q"].data_ptr(), dev["dhat"].data_ptr(),
                            dev["alpha2"].data_ptr(), eps=dev["eps"].data_ptr(), max_iters=20, sync=1)
        assert ei.value.code == smpc.SMPC_EDIVERGED, ei.value
        info = g.solve(20)  # the same factor solves again with finite data
        assert info["iterations"] == 20
    finally:
        g.close()
    _healthy_after()


def test_device_allocation_beyond_the_gpu_reports_enomem():
    import torch

    import paper_1604_01074_gb300 as smpc
    P = synth.barcelona(0)
    n = 2_000_001  # root + 2 million leaves
    parent = np.zeros(n, dtype=np.int32)
    parent[0] = -1
    total = torch.cuda.get_device_properties(0).total_memory
    tree = smpc.smpc_tree_create(parent)
    try:
        # float64 per-node packs: (177 x 98 + 97 x 98) entries, padded, of 8 bytes per node
        assert n * 26_912 * 8 > total
        with pytest.raises(smpc.SmpcError) as ei:
            smpc.smpc_factor(tree, P["net"], P["cost"], precision=0, lam=1e-3, schedule=2)
        assert ei.value.code == smpc.SMPC_ENOMEM, ei.value
    finally:
        smpc.smpc_tree_destroy(tree)
    _healthy_after()


def test_pipeline_wait_that_gives_up_reports_etimeout():
    import paper_1604_01074_gb300 as smpc
    P = synth.barcelona(0)
    tree, fac, _ = H.oracle_build(P)
    steps = H.closed_form_steps(fac, tree, 1e-6)
    os.environ["SMPC_PIPELINE_WAIT_NS"] = "0"
    try:
        g = H.Gpu(P, steps=steps, precision=1, schedule=2)
    finally:
        del os.environ["SMPC_PIPELINE_WAIT_NS"]
    try:
        with pytest.raises(smpc.SmpcError) as ei:
            g.solve(10)
        assert ei.value.code == smpc.SMPC_ETIMEOUT, ei.value
    finally:
        g.close()
    g = H.Gpu(P, steps=steps, precision=1, schedule=2)  # the normal bound again
    try:
        assert g.solve(10)["iterations"] == 10
    finally:
        g.close()
    _healthy_after()


def test_iteration_cap_beyond_the_limit_is_refused():
    import paper_1604_01074_gb300 as smpc
    P = synth.tiny(0)
    g = H.Gpu(P, steps=H.tiny_steps(P))
    try:
        with pytest.raises(smpc.SmpcError) as ei:
            smpc.smpc_solve(g.fac, P["p"], P["q"], P["dhat"], P["alpha2"], eps=P["eps"],
                            max_iters=smpc.SMPC_MAX_ITERS + 1, sync=1)
        assert ei.value.code == smpc.SMPC_EINVAL, ei.value
        with pytest.raises(smpc.SmpcError) as ei:
            smpc.smpc_profile_solve(g.fac, P["p"], P["q"], P["dhat"], P["alpha2"], eps=P["eps"], iters=4097)
        assert ei.value.code == smpc.SMPC_EINVAL, ei.value
        server = smpc.smpc_server_create(1 << 30, 1)
        try:
            with pytest.raises(smpc.SmpcError) as ei:
                smpc.smpc_submit(server, g.fac, P["p"], P["q"], P["dhat"], P["alpha2"], eps=P["eps"],
                                 max_iters=smpc.SMPC_MAX_ITERS + 1)
            assert ei.value.code == smpc.SMPC_EINVAL, ei.value
        finally:
            smpc.smpc_server_destroy(server)
        assert g.solve(20)["iterations"] == 20  # the factor is untouched
    finally:
        g.close()
    _healthy_after()
