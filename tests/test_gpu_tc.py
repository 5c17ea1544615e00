"""Parity of the tensor-core split-precision paths with the oracle and with the
FP64 GPU path.

Tolerances (normwise relative, over the compared entries):
 * TF32X3: each Khatri-Rao product z is split z = hi + lo with 11-bit parts, so
   the three products represent z_a z_b to about 2^-22 relative; the dropped
   lo*lo term is 2^-22 and the FP32 accumulation restarts every stage (4 hi*hi
   steps of at most 1 ulp truncation each) before an FP64 fold.  A simulation of
   the split alone gives relF ~1e-7; the bound used is 1e-6.
 * FP16X3: 11-bit parts as for TF32X3, on X~ scaled per variable by a power of
   two (exact, undone exactly on output), so the same bound applies.
 * BF16X3: 8-bit parts leave a 2^-16 relative representation error per product
   and a dropped lo*lo term that is biased on products of a column with itself,
   about 3e-6 relative in simulation; the bound used is 3e-5.
Orders whose entries nearly cancel (odd orders of symmetric data) are compared
relative to the tensor norm, which is dominated by the entries that do not;
single entries where a cumulant is a small difference of large moment terms
are compared against the moment scale.
"""
import numpy as np
import pytest

import blocks
import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = {1: 3e-5, 2: 1e-6, 3: 1e-6}   # by precision code


@pytest.fixture(scope="module")
def cum():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1701_05420_gb300 as m
    return m


def run(cum, X, d_max, b, prec):
    import torch
    Xt = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    ws = cum.workspace(X.shape[0], X.shape[1], d_max, b, prec)
    C, mean = cum.cumulants(Xt, d_max, b, prec, ws=ws)
    torch.cuda.synchronize()
    assert cum.cum_device_status(ws) == cum.CUM_OK
    return {d: v.cpu().numpy() for d, v in C.items()}


@pytest.mark.parametrize("prec", [1, 2, 3])
@pytest.mark.parametrize("t,n,b,dmax", [
    (3000, 10, 4, 4),    # several stages, ragged n
    (700, 7, 2, 6),      # orders up to 6, t below one t chunk
    (9000, 20, 4, 4),    # several tiles per order
    (130, 5, 5, 4),      # one block, t not a multiple of a stage
])
def test_small_full_tensor(cum, prec, t, n, b, dmax):
    X = synth.skewed(t, n, seed=2000 + t + n)
    C = run(cum, X, dmax, b, prec)
    for d in range(2, dmax + 1):
        ref = oracle.cumulant_dense(X, d)
        relF, relM = blocks.rel_errors(blocks.to_dense(C[d], n, d, b), ref)
        assert relF <= TOL[prec] and relM <= 4 * TOL[prec], (d, relF, relM)


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_matches_fp64_path(cum, prec):
    """Tiles across several row and column tiles, against the FP64 GPU path."""
    X = synth.skewed(20000, 40, seed=77).astype(np.float32)
    C64 = run(cum, X.astype(np.float64), 4, 4, 0)
    Ct = run(cum, X, 4, 4, prec)
    for d in (2, 3, 4):
        relF, relM = blocks.rel_errors(Ct[d], C64[d])
        assert relF <= TOL[prec] and relM <= 4 * TOL[prec], (d, relF, relM)


@pytest.mark.parametrize("prec", [2, 3])
def test_precision_workload_sampled(cum, prec):
    """t=1e6, n=128 skew-normal copula (float32), b=16, orders 2..3: FP16X3 and
    TF32X3 within 1e-6 of the oracle on sampled entries."""
    X = synth.precision()
    C = run(cum, X, 3, 16, prec)
    _, Xc = oracle.center(X.astype(np.float64))
    for d in (2, 3):
        idx = synth.sample_indices(128, d, 400, seed=40 + d)
        ref = oracle.cumulant_entries(Xc, idx)
        got = C[d][blocks.entry_offsets(idx, 128, 16)]
        relF, relM = blocks.rel_errors(got, ref)
        assert relF <= TOL[prec] and relM <= TOL[prec], (d, relF, relM)


@pytest.fixture(scope="module")
def high_order(cum):
    """The high-order workload (t=2e5, n=48 Laplace x orthogonal mix, float32,
    b=4): its FP64-centred copy for the oracle, and its cumulants of orders 2..6
    on the FP64 GPU path, which tests/test_gpu_fp64.py holds within 1e-10 of the
    oracle on this workload."""
    X = synth.high_order()
    _, Xc = oracle.center(X.astype(np.float64))
    C64 = run(cum, X.astype(np.float64), 6, 4, 0)
    return X, Xc, C64


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_high_order_full_tensor(cum, high_order, prec):
    """Every stored entry of orders 2..6 against the FP64 path: the normwise
    error of the whole tensor (relF) within the split tolerance."""
    X, _, C64 = high_order
    C = run(cum, X, 6, 4, prec)
    for d in range(2, 7):
        relF, relM = blocks.rel_errors(C[d], C64[d])
        assert relF <= TOL[prec], (d, relF, relM)


def _specials(n, d):
    """Multi-indices with few distinct variables (all equal, two or three
    values repeated), where the moments and the partition products cancel most:
    on this data |M| / |C| reaches about 60 at order 6."""
    idx = []
    for v in (0, n // 2, n - 1):
        idx.append([v] * d)
    for a, c in ((0, n - 1), (3, 17), (n // 2, 5)):
        idx.append([a] * (d - d // 2) + [c] * (d // 2))
    for a, c, e in ((1, 20, 40), (7, 8, 9)):
        idx.append(([a, c, e] * d)[:d])
    return np.asarray(idx, dtype=np.int32)


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_high_order_sampled(cum, high_order, prec):
    """Orders 2..6 against the oracle (Eq. cumfmom).  Uniformly sampled
    multi-indices: relF and relMax within the split tolerance.  Entries with few
    distinct variables, where the cumulant is a small difference of large
    moment and partition terms: their error within the tolerance relative to the
    moments they are computed from (the cancellation itself is the data's)."""
    X, Xc, _ = high_order
    C = run(cum, X, 6, 4, prec)
    for d in range(2, 7):
        idx = synth.sample_indices(48, d, 300, seed=50 + d, include_special=False)
        ref = oracle.cumulant_entries(Xc, idx)
        got = C[d][blocks.entry_offsets(idx, 48, 4)]
        relF, relM = blocks.rel_errors(got, ref)
        assert relF <= TOL[prec] and relM <= TOL[prec], (d, relF, relM)
        sp = _specials(48, d)
        refC = oracle.cumulant_entries(Xc, sp)
        refM = oracle.moment_entries(Xc, sp)
        gotS = C[d][blocks.entry_offsets(sp, 48, 4)]
        err = np.linalg.norm(gotS - refC) / np.linalg.norm(refM)
        assert err <= TOL[prec], (d, err)


@pytest.mark.parametrize("prec", [1, 2, 3])
@pytest.mark.parametrize("t,n,b,dmax", [
    (5000, 200, 8, 3),    # 200 variables: 200-row TMA boxes, shallow rings
    (3000, 256, 16, 2),   # the widest staged operand (256 variables)
    (4000, 65, 1, 3),     # b = 1 with a ragged 65-row box
])
def test_wide_and_degenerate_shapes(cum, prec, t, n, b, dmax):
    X = synth.skewed(t, n, seed=3000 + n).astype(np.float32)
    C = run(cum, X, dmax, b, prec)
    C64 = run(cum, X.astype(np.float64), dmax, b, 0)
    for d in range(2, dmax + 1):
        relF, relM = blocks.rel_errors(C[d], C64[d])
        assert relF <= TOL[prec] and relM <= 4 * TOL[prec], (d, relF, relM)


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_columns_of_very_different_scale(cum, prec):
    """Columns scaled by 1e-6 .. 1e6: the fp16 parts rely on the per-variable
    power-of-two scaling to stay in range.  Errors are measured on the
    standardised tensor C[i1..id] / (s_i1 ... s_id), s = column std."""
    n, b, dmax = 12, 3, 4
    X = (synth.skewed(8000, n, seed=4242) * 10.0 ** np.linspace(-6, 6, n)).astype(np.float32)
    C = run(cum, X, dmax, b, prec)
    C64 = run(cum, X.astype(np.float64), dmax, b, 0)
    sd = X.astype(np.float64).std(axis=0)
    for d in range(2, dmax + 1):
        S = sd
        for _ in range(d - 1):
            S = np.multiply.outer(S, sd)
        got = blocks.to_dense(C[d], n, d, b) / S
        ref = blocks.to_dense(C64[d], n, d, b) / S
        relF, relM = blocks.rel_errors(got, ref)
        assert relF <= TOL[prec] and relM <= 4 * TOL[prec], (d, relF, relM)
