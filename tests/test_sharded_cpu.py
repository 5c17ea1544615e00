"""The t-sharded driver (Alg. 3 across processes) with world_size 2 over gloo
on CPU.  The compute steps are a numpy stand-in working on each process's
shard only; the test checks the exchange logic: shard boundaries, the global
two-pass mean, the global residual means of the stored shards, and sums
exchanged before the division by the global t."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth


class NumpyShardOps:
    """Stand-in compute steps on one shard (moments only: finalize scales).

    Its stored centred shard carries a per-column offset delta, as the split
    precisions' FP32 rounding leaves a residual mean: the moment sums are taken
    about the residual mean set by set_residual_sums, so the result matches the
    oracle only if every shard uses the global residual means."""

    DELTA = np.array([1e-3, -2e-3, 5e-4, 3e-3])

    def __init__(self):
        self.Xc = None
        self.m = None

    def column_sums(self, X, shift):
        X = X.numpy()
        s = shift.numpy() if shift is not None else 0.0
        return torch.from_numpy((X - s).sum(axis=0))

    def mean_from_sums(self, t_total, shift, sums):
        s = shift if shift is not None else 0.0
        return s + sums / t_total

    def center_with_mean(self, X, mean):
        self.Xc = X.numpy() - mean.numpy() + self.DELTA[: X.shape[1]]
        self.m = self.Xc.sum(axis=0) / self.Xc.shape[0]   # the shard's own residual mean until replaced

    def residual_sums(self):
        return torch.from_numpy(self.Xc.sum(axis=0))

    def set_residual_sums(self, sums, t_total):
        self.m = sums.numpy() / t_total

    def moment_sums(self, d):
        t = self.Xc.shape[0]
        return torch.from_numpy(np.ascontiguousarray(oracle.moment_dense(self.Xc - self.m, d) * t))

    def finalize(self, d, scale, S, lower):
        return S * scale


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, X, d_max, out_q):
    from paper_1701_05420_gb300.sharded import shard_rows, sharded_cumulants
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lo, hi = shard_rows(X.shape[0], world, rank)
    Xl = torch.from_numpy(X[lo:hi].copy())
    C, mean = sharded_cumulants(Xl, X.shape[0], d_max, lambda x: dist.all_reduce(x), NumpyShardOps())
    out_q.put((rank, {d: v.numpy() for d, v in C.items()}, mean.numpy()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("t", [1001, 64])
def test_two_rank_gloo_exchange(t):
    pytest.importorskip("paper_1701_05420_gb300")
    X = synth.skewed(t, 4, seed=123) + 1e3
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, X, 4, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    mu, Xc = oracle.center(X)
    for rank, C, mean in results:
        np.testing.assert_allclose(mean, mu, rtol=1e-14)
        for d in (2, 3, 4):
            ref = oracle.moment_dense(Xc, d)
            np.testing.assert_allclose(C[d], ref, rtol=0, atol=1e-11 * np.abs(ref).max())


def test_shard_rows_partition():
    from paper_1701_05420_gb300.sharded import shard_rows
    for t in (1, 7, 100, 1001):
        for world in (1, 2, 3, 8):
            ranges = [shard_rows(t, world, r) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == t
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            sizes = [h - l for l, h in ranges]
            assert max(sizes) - min(sizes) <= 1
