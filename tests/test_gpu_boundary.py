"""The C ABI used call by call, the way a caller strings the steps together,
on the high-order workload (t = 200000, n = 48 Laplace x orthogonal mix,
float32, b = 4) where every order's plan splits the sample axis (Alg. 3):

 * cum_center once, then cum_moment_blocks for each order 2..6 on the same
   workspace (Alg. 1-2 after Def. 1.3): sampled moment entries against the
   oracle's Eq. d::moment;
 * the t-sharded steps (cum_column_sums ... cum_finalize, Alg. 3 / Eq. mapred)
   over two shards large enough that each shard's plan splits too: sampled
   cumulant entries against the oracle's Eq. cumfmom.

cum_center lays its workspace out for order 2 and cum_moment_blocks for its
own order, so these tests fail if any region centring writes moves with the
order.  cum_moment_blocks also applies the residual-mean correction on split
precisions, and the sharded steps exchange the stored data's residual sums.
Tolerances are those of the split-precision paths (normwise over the sampled
entries, plus the largest entry error against the largest entry; cumulant
entries with few distinct variables against the moments they cancel)."""
import numpy as np
import pytest

import blocks
import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 2: 1e-6, 3: 1e-6}
SAMPLES = 300


@pytest.fixture(scope="module")
def cum():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1701_05420_gb300 as m
    return m


@pytest.fixture(scope="module")
def data():
    X = synth.high_order()
    _, Xc = oracle.center(X.astype(np.float64))
    return X, Xc


@pytest.mark.parametrize("prec", [2, 3])
def test_center_then_moment_blocks_every_order(cum, data, prec):
    import torch
    X, Xc = data
    t, n, b = X.shape[0], X.shape[1], 4
    for d in range(3, 6):   # the sample axis is split at these orders
        assert cum.cum_plan_info(d, t, n, b, prec)["splits"] > 1, d
    ws = cum.workspace(t, n, 6, b, prec)
    Xt = torch.from_numpy(X).cuda()
    cum.cum_center(Xt, b, prec, None, ws)
    for d in range(2, 7):
        M = torch.full((cum.num_entries(n, d, b),), float("nan"), dtype=torch.float64, device="cuda")
        cum.cum_moment_blocks(d, t, n, b, prec, M, ws)
        torch.cuda.synchronize()
        assert cum.cum_device_status(ws) == cum.CUM_OK
        idx = synth.sample_indices(n, d, SAMPLES, seed=700 + d)
        ref = oracle.moment_entries(Xc, idx)
        got = M.cpu().numpy()[blocks.entry_offsets(idx, n, b)]
        relF, relM = blocks.rel_errors(got, ref)
        assert relF <= TOL[prec] and relM <= TOL[prec], (d, relF, relM)


@pytest.mark.parametrize("prec", [0, 2, 3])
def test_sharded_steps_with_split_shards(cum, data, prec):
    import torch

    from paper_1701_05420_gb300.sharded import LibraryOps, shard_rows
    X, Xc = data
    t, n, b, dmax = X.shape[0], X.shape[1], 4, 5
    Xin = X.astype(np.float64) if prec == 0 else X
    shards = [shard_rows(t, 2, r) for r in range(2)]
    for lo, hi in shards:
        assert cum.cum_plan_info(4, hi - lo, n, b, prec)["splits"] > 1
    Xs = [torch.from_numpy(np.ascontiguousarray(Xin[lo:hi])).cuda() for lo, hi in shards]
    ops = [LibraryOps(hi - lo, n, dmax, b, prec, "cuda") for lo, hi in shards]
    # the two shards in lock-step; each exchange sums both shards' tensors
    s1 = [o.column_sums(x, None) for o, x in zip(ops, Xs)]
    tot = s1[0] + s1[1]
    m1 = [o.mean_from_sums(t, None, tot) for o in ops]
    s2 = [o.column_sums(x, m) for o, x, m in zip(ops, Xs, m1)]
    tot2 = s2[0] + s2[1]
    mean = [o.mean_from_sums(t, m, tot2) for o, m in zip(ops, m1)]
    for o, x, m in zip(ops, Xs, mean):
        o.center_with_mean(x, m)
    r = [o.residual_sums() for o in ops]
    rtot = r[0] + r[1]
    for o in ops:
        o.set_residual_sums(rtot, t)
    C = {}
    for d in range(2, dmax + 1):
        S = [o.moment_sums(d) for o in ops]
        C[d] = ops[0].finalize(d, 1.0 / t, S[0] + S[1], [C[k] for k in range(2, d - 1)])
    torch.cuda.synchronize()
    mu, _ = oracle.center(X.astype(np.float64))
    np.testing.assert_allclose(mean[0].cpu().numpy(), mu, rtol=1e-13, atol=1e-12)
    for d in range(2, dmax + 1):
        # uniform multi-indices: relF and relMax within the tolerance
        idx = synth.sample_indices(n, d, SAMPLES, seed=800 + d, include_special=False)
        ref = oracle.cumulant_entries(Xc, idx)
        got = C[d].cpu().numpy()[blocks.entry_offsets(idx, n, b)]
        relF, relM = blocks.rel_errors(got, ref)
        assert relF <= TOL[prec] and relM <= TOL[prec], (d, relF, relM)
        # entries with few distinct variables, where the cumulant is a small
        # difference of large terms: error relative to the moments they come from
        sp = synth.sample_indices(n, d, 8, seed=900 + d)[:6]
        refC = oracle.cumulant_entries(Xc, sp)
        refM = oracle.moment_entries(Xc, sp)
        gotS = C[d].cpu().numpy()[blocks.entry_offsets(sp, n, b)]
        assert np.linalg.norm(gotS - refC) <= TOL[prec] * np.linalg.norm(refM), d
