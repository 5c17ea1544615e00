"""The step entry points of the t-sharded path on one GPU: two shards of one
dataset go through column sums, the global two-pass mean, centring with that
mean, unnormalised moment sums and the finalisation; the exchange is a sum of
the two shards' tensors (column sums, the stored shards' residual sums, and
the moment sums).  Result must equal cum_cumulants on the whole data."""
import numpy as np
import pytest

import blocks
import synth
from paper_1701_05420_gb300.sharded import shard_rows, sharded_cumulants

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cum():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1701_05420_gb300 as m
    return m


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (3, 1e-6), (2, 1e-6)])
def test_two_shards_equal_whole(cum, prec, tol):
    import torch
    from paper_1701_05420_gb300.sharded import LibraryOps
    t, n, b, dmax = 5003, 9, 3, 5
    X = synth.skewed(t, n, seed=321).astype(np.float64 if prec == 0 else np.float32)
    whole, _ = cum.cumulants(torch.from_numpy(X).cuda(), dmax, b, prec)

    shards = [shard_rows(t, 2, r) for r in range(2)]
    Xs = [torch.from_numpy(np.ascontiguousarray(X[lo:hi])).cuda() for lo, hi in shards]
    ops = [LibraryOps(hi - lo, n, dmax, b, prec, "cuda") for lo, hi in shards]

    # the two shards in lock-step; each exchange is the sum of both shards' tensors
    s1 = [o.column_sums(x, None) for o, x in zip(ops, Xs)]
    tot = s1[0] + s1[1]
    m1 = [o.mean_from_sums(t, None, tot) for o in ops]
    s2 = [o.column_sums(x, m) for o, x, m in zip(ops, Xs, m1)]
    tot2 = s2[0] + s2[1]
    mean = [o.mean_from_sums(t, m, tot2) for o, m in zip(ops, m1)]
    for o, x, m in zip(ops, Xs, mean):
        o.center_with_mean(x, m)
    # the stored shards' residual column sums, exchanged (split precisions)
    r = [o.residual_sums() for o in ops]
    rtot = r[0] + r[1]
    for o in ops:
        o.set_residual_sums(rtot, t)
    C = [{}, {}]
    for d in range(2, dmax + 1):
        S = [o.moment_sums(d) for o in ops]
        Ssum = S[0] + S[1]
        for r in range(2):
            Sr = Ssum.clone()
            C[r][d] = ops[r].finalize(d, 1.0 / t, Sr, [C[r][k] for k in range(2, d - 1)])
    torch.cuda.synchronize()
    for r in range(2):
        for d in range(2, dmax + 1):
            relF, relM = blocks.rel_errors(C[r][d].cpu().numpy(), whole[d].cpu().numpy())
            assert relF <= tol and relM <= tol, (r, d, relF, relM)


def test_single_process_driver(cum):
    """sharded_cumulants with one process (allreduce = identity) equals cum_cumulants."""
    import torch
    from paper_1701_05420_gb300.sharded import LibraryOps
    t, n, b, dmax = 4000, 7, 2, 6
    X = torch.from_numpy(synth.skewed(t, n, seed=9)).cuda()
    C, mean = sharded_cumulants(X, t, dmax, lambda x: None, LibraryOps(t, n, dmax, b, 0, "cuda"))
    whole, mean2 = cum.cumulants(X, dmax, b, 0)
    torch.cuda.synchronize()
    for d in range(2, dmax + 1):
        relF, relM = blocks.rel_errors(C[d].cpu().numpy(), whole[d].cpu().numpy())
        assert relF <= 1e-12, (d, relF)


@pytest.mark.parametrize("prec", [2, 3])
def test_shard_without_global_residual_is_uncorrected(cum, prec):
    """A shard centred by a global mean keeps its own column sums, which hold
    its deviation from that mean: until cum_set_residual_sums supplies the
    global sums its moment sums carry no residual-mean correction (they equal
    the raw contraction), rather than a correction by the shard's own mean."""
    import torch
    from paper_1701_05420_gb300.sharded import LibraryOps
    t, n, b, d = 6000, 9, 3, 3
    X = torch.from_numpy(synth.skewed(t, n, seed=77).astype(np.float32)).cuda()
    ops = LibraryOps(t // 2, n, d, b, prec, "cuda")
    mean = X.double().mean(dim=0)          # the mean of all rows, not of this half
    half = X[: t // 2].contiguous()
    ops.center_with_mean(half, mean)
    S = ops.moment_sums(d)
    raw = torch.empty_like(S)
    cum.cum_moment_contraction(d, t // 2, n, b, prec, raw, ops.ws)   # moments: the sums / (t/2)
    torch.cuda.synchronize()
    rel = ((S / (t // 2) - raw).norm() / raw.norm()).item()
    assert rel < 1e-14, rel
