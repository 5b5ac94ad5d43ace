"""One scenario tree split over several GPUs: the host loop of a sharded solve.

Each process (one per GPU) owns a contiguous range of the tree's chains and replicates
the top nodes above them (smpc_shard_* in the C ABI, Sec. IV-B's stage parallelism
across GPUs).  Every APG iteration does two exchanges through torch.distributed:

* allreduce (sum) of the per-cut-parent sums of s and r over each GPU's chain heads,
  between the local half and the top half of the backward sweep;
* allreduce (max) of the iteration's residual triple (rho, ||Hz||, ||t||), so that every
  GPU takes the same stop decision from the same numbers.

The exchange runs on device tensors with NCCL (stream-ordered on the current stream)
and through host memory with gloo.  ``sharded_solve`` drives any object with the
methods of ``LibraryShard`` (begin, local, top, tail, flags, finish and the tensors
``exchange`` and ``residuals``), so the same host code serves the library and other
implementations of the phases.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def chain_range(n_chains, rank, world):
    """Contiguous chains [begin, end) of `rank` out of `world`, balanced to within one."""
    base, extra = divmod(n_chains, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def _allreduce(t, op, group):
    if t.is_cuda and dist.get_backend(group) == "nccl":
        dist.all_reduce(t, op=op, group=group)
        return
    host = t.cpu()
    dist.all_reduce(host, op=op, group=group)
    t.copy_(host)


def sharded_solve(shard, step, group=None, max_iters=500, tol=0.0, check_every=32):
    """Runs the solve of `shard` in lockstep with the other ranks of `group`; returns
    the result dict of shard.finish.  Every rank must call it with the same settings."""
    shard.begin(step, max_iters, tol)
    launched = 0
    for nu in range(max_iters):
        shard.local(nu)
        _allreduce(shard.exchange, dist.ReduceOp.SUM, group)
        shard.top(nu)
        if nu >= 1:  # the residual of iteration nu - 1, written by this iteration's prox
            _allreduce(shard.residuals[3 * (nu - 1):3 * nu], dist.ReduceOp.MAX, group)
        launched = nu + 1
        if check_every and launched % check_every == 0:
            done, err = shard.flags()
            if done >= 0 or err:
                break
    shard.tail(launched)
    if launched >= 1:
        _allreduce(shard.residuals[3 * (launched - 1):3 * launched], dist.ReduceOp.MAX, group)
    return shard.finish(launched)


class LibraryShard:
    """This GPU's shard of a factor through the C ABI (smpc_shard_*)."""

    def __init__(self, fac, precision, chain_begin, chain_end, n_nodes, n_x, n_u, device=None):
        import paper_1604_01074_gb300 as smpc
        self.smpc = smpc
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.h = smpc.smpc_shard_create(fac, chain_begin, chain_end)
        self.n_cut, self.width, self.n_local = smpc.smpc_shard_info(self.h)
        self.nodes = smpc.smpc_shard_nodes(self.h)  # the rows this shard's outputs hold
        self.dtype = torch.float64 if precision == 0 else torch.float32
        self.exchange = torch.zeros((max(self.n_cut, 1), self.width), dtype=self.dtype, device=self.device)
        self.residuals = None
        dt = self.dtype
        self.u = torch.zeros((n_nodes, n_u), dtype=dt, device=self.device)
        self.x = torch.zeros((n_nodes, n_x), dtype=dt, device=self.device)
        self.y = torch.zeros((n_nodes, 2 * n_x + n_u), dtype=dt, device=self.device)

    def begin(self, step, max_iters, tol):
        # float64 bit patterns of non-negative numbers order as int64: MAX works on them
        self.residuals = torch.zeros(3 * (max_iters + 2), dtype=torch.int64, device=self.device)
        self.smpc.smpc_shard_begin(self.h, step["p"], step["q"], step["dhat"], step["alpha2"],
                                   self.residuals.data_ptr(), eps=step.get("eps"), max_iters=max_iters, tol=tol,
                                   stream=torch.cuda.current_stream(self.device))

    def local(self, nu):
        self.smpc.smpc_shard_step(self.h, nu, 0, self.exchange.data_ptr())

    def top(self, nu):
        self.smpc.smpc_shard_step(self.h, nu, 1, self.exchange.data_ptr())

    def tail(self, n):
        self.smpc.smpc_shard_step(self.h, n, 2)

    def flags(self):
        return self.smpc.smpc_shard_flags(self.h)

    def finish(self, launched):
        return self.smpc.smpc_shard_finish(self.h, launched, u=self.u, x=self.x, y=self.y)

    def close(self):
        self.smpc.smpc_shard_destroy(self.h)
