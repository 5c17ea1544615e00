"""Cumulants of a dataset whose samples are split across processes (Alg. 3).

Each process holds a contiguous shard of the rows of X.  The exchange steps
are the sums the method needs across shards: the column sums of the centring
(Def. 1.3; two passes, the second on the residual of the first mean), the
column sums of the stored centred data (on split precisions order 6 reads
X~ rounded to FP32, whose small residual mean is removed from those moments
to first order) and
the unnormalised moment sums of every order (Eq. momentp1).  After the
moment sums are exchanged, every process divides by the global t and applies
the cumulant correction (Eq. cum_r), so all processes end with the same
cumulant tensors.

The compute steps are the library's C ABI calls (``LibraryOps``); the exchange
is an ``allreduce(tensor)`` callable that sums in place (for example
``torch.distributed.all_reduce`` over NCCL).  ``ops`` can be replaced to run
this driver's exchange logic without a GPU.
"""
from __future__ import annotations


class LibraryOps:
    """The compute steps, on the GPU, through the C ABI."""

    def __init__(self, t_local, n, d_max, b, prec, device):
        import torch

        import paper_1701_05420_gb300 as cum
        self.cum, self.torch = cum, torch
        self.t, self.n, self.b, self.prec, self.device = t_local, n, b, prec, device
        self.ws = cum.workspace(t_local, n, d_max, b, prec, device)

    def zeros_vec(self):
        return self.torch.zeros(self.n, dtype=self.torch.float64, device=self.device)

    def column_sums(self, X, shift):
        out = self.zeros_vec()
        self.cum.cum_column_sums(X, self.b, self.prec, shift, out, self.ws)
        return out

    def mean_from_sums(self, t_total, shift, sums):
        out = self.zeros_vec()
        self.cum.cum_mean_from_sums(self.n, t_total, shift, sums, out)
        return out

    def center_with_mean(self, X, mean):
        self.cum.cum_center_with_mean(X, self.b, self.prec, mean, self.ws)

    def residual_sums(self):
        out = self.zeros_vec()
        self.cum.cum_residual_sums(self.n, self.b, self.prec, out, self.ws)
        return out

    def set_residual_sums(self, sums, t_total):
        self.cum.cum_set_residual_sums(self.n, self.b, self.prec, sums, t_total, self.ws)

    def moment_sums(self, d):
        out = self.torch.empty(self.cum.num_entries(self.n, d, self.b), dtype=self.torch.float64,
                               device=self.device)
        self.cum.cum_moment_sums(d, self.t, self.n, self.b, self.prec, out, self.ws)
        return out

    def finalize(self, d, scale, S, lower):
        self.cum.cum_finalize(d, self.n, self.b, scale, S, lower, S)
        return S


def sharded_cumulants(X_local, t_total, d_max, allreduce, ops):
    """Cumulants of orders 2..d_max of the rows of all shards.

    X_local: this process's rows; t_total: rows over all processes;
    allreduce(x): in-place sum of a tensor over processes.  Returns
    ({d: block tensor}, mean)."""
    s1 = ops.column_sums(X_local, None)
    allreduce(s1)
    m1 = ops.mean_from_sums(t_total, None, s1)
    s2 = ops.column_sums(X_local, m1)
    allreduce(s2)
    mean = ops.mean_from_sums(t_total, m1, s2)
    ops.center_with_mean(X_local, mean)
    # the stored centred shards keep residual column means (FP32 rounding of
    # X - mean on split precisions); every shard corrects with the global ones
    r = ops.residual_sums()
    allreduce(r)
    ops.set_residual_sums(r, t_total)
    C = {}
    for d in range(2, d_max + 1):
        S = ops.moment_sums(d)
        allreduce(S)
        C[d] = ops.finalize(d, 1.0 / t_total, S, [C[k] for k in range(2, d - 1)])
    return C, mean


def shard_rows(t, world, rank):
    """Contiguous row range [lo, hi) of `rank` among `world` processes (Alg. 3;
    the last shards take one row less when world does not divide t)."""
    base, extra = divmod(t, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)
