"""Reduced precision (float32 and bfloat16 packs) against the FP64 oracle, element by
element, at full size: the 2081-node tree (100 scenarios) on every schedule with
per-node packs, with shared packs, and samples of the 21 111-node tree (1000
scenarios) that reach the widest tensor-core GEMM of the bfloat16 shared-pack launch.

Bars (max over u, x, y of |gpu - oracle| / (1 + |oracle|_inf), at equal iteration
counts; the oracle runs the same steps):

* float32 packs, FP32_BOUND = 1e-4.  Every vector entry is rounded to float32
  (unit roundoff 2^-24 = 6e-8) and the mat-vecs accumulate up to n_x + n_u = 177
  products in float32; the subtree sums of Algorithm 1 then add up to 2081 (21 111)
  such terms, whose rounding errors grow at most linearly in the count of terms, so
  errors of 1e-5 relative to the largest entry are the expected size, and 1e-4 keeps
  a margin of ten.  The dual state is carried in float-float (48 bits) and adds nothing.
* bfloat16 packs (anchored every 16 iterations), BF16_BOUND = 2e-3.  Between anchors
  the solve step applies bfloat16 matrices (unit roundoff 2^-9 = 2e-3) to w - w_a, the
  change of w since the last anchor, while the part at the anchor is float32; the
  error is a fraction of 2^-9 of that change, which is smaller than the largest
  entry, so 2^-9 relative to the largest entry bounds it.

Besides: |rho_rel,gpu - rho_rel,oracle| <= 1e-4 (the reduced-precision tolerance) and
the demand coupling |E u + E_d d| of the float32 result, which the oracle satisfies to
1e-12, to float32 rounding of the largest input.
"""
import numpy as np
import pytest

import synth
from tests import harness as H

pytestmark = pytest.mark.gpu

FP32_BOUND = 1e-4
BF16_BOUND = 2e-3
RHO_TOL = 1e-4
BOUND = {1: FP32_BOUND, 2: BF16_BOUND}

_ORACLE = {}


def _oracle(P, steps, iters):
    key = (P["name"], iters)
    if key not in _ORACLE:
        _ORACLE[key] = H.oracle_run(P, steps, iters)
    return _ORACLE[key]


def _compare(P, steps, iters, precision, schedule=0, shared_packs=0):
    R = _oracle(P, steps, iters)
    g = H.Gpu(P, steps=steps, precision=precision, schedule=schedule, shared_packs=shared_packs)
    try:
        info = g.solve(iters)
        used = g.smpc.smpc_factor_schedule(g.fac)[0]
        u, x, y = g.arrays()
    finally:
        g.close()
    assert info["iterations"] == iters
    if schedule:
        assert used == schedule
    eu, ex, ey = H.relerr(u, R.u), H.relerr(x, R.x), H.relerr(y, H.stack_y(R.y))
    drho = abs(info["rho_rel"] - R.rho_rel[-1])
    cpl = H.coupling_residual(P, u)
    msg = dict(precision=precision, schedule=used, shared=shared_packs, iters=iters, eu=eu, ex=ex, ey=ey,
               drho=drho, coupling=cpl, rho_rel=info["rho_rel"])
    print("reduced-parity", msg)
    assert max(eu, ex, ey) <= BOUND[precision], msg
    assert drho <= RHO_TOL, msg
    # the oracle meets the coupling to 1e-12; float32 rounding of inputs up to max |u|
    assert cpl <= 1e-5 * (1.0 + np.abs(R.u).max()) * (1 if precision == 1 else 10), msg
    return msg


@pytest.fixture(scope="module")
def barcelona_case():
    P = synth.barcelona(0)
    return P, H.full_size_steps(P)


@pytest.mark.parametrize("iters", [10, 60])
@pytest.mark.parametrize("schedule", [1, 2, 3])
@pytest.mark.parametrize("precision", [1, 2])
def test_per_node_packs_full_size(barcelona_case, precision, schedule, iters):
    P, steps = barcelona_case
    _compare(P, steps, iters, precision, schedule=schedule)


@pytest.mark.parametrize("iters", [10, 60])
@pytest.mark.parametrize("precision", [1, 2])
def test_shared_packs_full_size(barcelona_case, precision, iters):
    P, steps = barcelona_case
    _compare(P, steps, iters, precision, shared_packs=1)


@pytest.fixture(scope="module")
def large_case():
    P = synth.large(0)
    return P, H.full_size_steps(P, power_iters=30)


@pytest.mark.parametrize("precision,shared", [(1, 0), (2, 0), (2, 1)])
def test_large_tree_sample(large_case, precision, shared):
    """30 iterations on the 21 111-node tree (1000 scenarios): float32 and bfloat16
    per-node packs on the schedule the factor picks by timing (the bench's launch
    configuration), and bfloat16 shared packs, whose delta launches run the Lambda and
    [Bbar; L] products on the tensor cores as 64-node GEMMs (a tree this size gives
    every SM at least two 32-node batches, so the launch takes its widest GEMM)."""
    P, steps = large_case
    assert len(P["tree"]["parent"]) == 21111
    _compare(P, steps, 30, precision, shared_packs=shared)
