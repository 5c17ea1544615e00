"""Parity of the FP64 GPU path (CUM_PREC_FP64) with the oracle.

Tolerance: the normwise relative error relF = ||C_gpu - C_ref||_F / ||C_ref||_F
over the compared entries must be <= 1e-10 (FP64 path target), and every entry
must be within 1e-10 * max|C_ref|.
"""
import numpy as np
import pytest

import blocks
import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def cum():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1701_05420_gb300 as m
    return m


def run(cum, X, d_max, b, prec=0, dtype="f64"):
    import torch
    Xt = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float64 if dtype == "f64" else np.float32)).cuda()
    C, mean = cum.cumulants(Xt, d_max, b, prec)
    torch.cuda.synchronize()
    return {d: v.cpu().numpy() for d, v in C.items()}, mean.cpu().numpy()


def check(got, ref, tol=TOL):
    relF, relM = blocks.rel_errors(got, ref)
    assert relF <= tol and relM <= tol, (relF, relM)
    return relF, relM


def test_paper_small_full_tensor(cum):
    """t=2000, n=20, b=4, orders 2..4: every entry against the full-tensor oracle."""
    X = synth.paper_small()
    C, mean = run(cum, X, 4, 4)
    mu, _ = oracle.center(X)
    np.testing.assert_allclose(mean, mu, rtol=1e-14, atol=1e-13)
    for d in (2, 3, 4):
        ref = oracle.cumulant_dense(X, d)
        check(blocks.to_dense(C[d], 20, d, 4), ref)
        # the stored blocks themselves, including diagonal-block duplicates
        check(C[d], blocks.from_dense(ref, 20, d, 4))


@pytest.mark.parametrize("t,n,b,dmax", [
    (37, 7, 3, 4),      # ragged n (padding) and a t far below one chunk
    (5, 3, 1, 4),       # b = 1: every block is one entry
    (300, 5, 5, 4),     # b = n: a single (diagonal) block
    (1000, 6, 8, 3),    # b > n: one padded block
    (129, 6, 2, 6),     # orders up to 6, t not a multiple of any step
    (2500, 9, 2, 5),    # several t chunks, ragged last block
    (1, 4, 2, 4),       # one sample: centred data is zero
    (4100, 13, 4, 4),   # t just above a chunk boundary, ragged n
])
def test_edge_shapes(cum, t, n, b, dmax):
    X = synth.skewed(t, n, seed=1000 + t + n)
    C, _ = run(cum, X, dmax, b)
    for d in range(2, dmax + 1):
        ref = oracle.cumulant_dense(X, d)
        got = blocks.to_dense(C[d], n, d, b)
        if np.abs(ref).max() == 0:
            assert np.abs(got).max() == 0
        else:
            check(got, ref)


def test_float32_input(cum):
    X = synth.skewed(3000, 10, seed=7).astype(np.float32)
    C, _ = run(cum, X, 4, 3, dtype="f32")
    for d in (2, 3, 4):
        check(blocks.to_dense(C[d], 10, d, 3), oracle.cumulant_dense(X.astype(np.float64), d))


def test_moment_blocks_alone(cum):
    import torch
    X = synth.skewed(1500, 11, seed=8)
    Xt = torch.from_numpy(X).cuda()
    M = cum.moments(Xt, (2, 3, 4, 5), b=3)
    _, Xc = oracle.center(X)
    for d, v in M.items():
        check(blocks.to_dense(v.cpu().numpy(), 11, d, 3), oracle.moment_dense(Xc, d))


def test_correct_alone(cum):
    """Alg. 4-5 in isolation: oracle moments and lower cumulants in, cumulant out."""
    import torch
    X = synth.skewed(800, 7, seed=9)
    n, b = 7, 2
    _, Xc = oracle.center(X)
    Cref = {d: oracle.cumulant_dense(X, d) for d in range(2, 7)}
    for d in (4, 5, 6):
        M = torch.from_numpy(blocks.from_dense(oracle.moment_dense(Xc, d), n, d, b)).cuda()
        low = [torch.from_numpy(blocks.from_dense(Cref[k], n, k, b)).cuda() for k in range(2, d - 1)]
        out = torch.empty_like(M)
        cum.cum_correct(d, n, b, M, low, out)
        torch.cuda.synchronize()
        check(out.cpu().numpy(), blocks.from_dense(Cref[d], n, d, b))


@pytest.mark.parametrize("b", [3, 5, 6])
def test_order6_correction_paths(cum, b):
    """Order-6 correction through each launch form: lower-order blocks staged in
    shared memory with one (b = 3) or three (b = 5) looped leading digits, and
    the general kernel (b = 6, whose staged blocks would exceed shared memory)."""
    n = 7
    X = synth.skewed(240, n, seed=600 + b)
    C, _ = run(cum, X, 6, b)
    for d in (4, 5, 6):
        check(blocks.to_dense(C[d], n, d, b), oracle.cumulant_dense(X, d))


@pytest.mark.parametrize("b", [2, 3, 4, 5, 6])
def test_order6_moment_form_matches_partition_form(cum, b):
    """cum_correct_m4 (order-4 moments in place of the three-pair partitions)
    against cum_correct (all 40 partitions) on the same moments and lower-order
    cumulants: staged with 0-3 looped digits (b = 2..5) and the general kernel
    (b = 6), which ignores M_4."""
    import torch
    n, t = 9, 3000
    X = torch.from_numpy(synth.skewed(t, n, seed=650 + b)).cuda()
    C, _ = cum.cumulants(X, 4, b, 0)
    ws = cum.workspace(t, n, 6, b, 0)
    cum.cum_center(X, b, 0, None, ws)
    M = {d: torch.empty(cum.num_entries(n, d, b), dtype=torch.float64, device="cuda") for d in (4, 6)}
    for d in (4, 6):
        cum.cum_moment_blocks(d, t, n, b, 0, M[d], ws)
    low = [C[2], C[3], C[4]]
    ref = torch.empty_like(M[6])
    got = torch.empty_like(M[6])
    cum.cum_correct(6, n, b, M[6], low, ref)
    cum.cum_correct_m4(n, b, M[6], low, M[4], got)
    torch.cuda.synchronize()
    check(got.cpu().numpy(), ref.cpu().numpy(), tol=1e-11)
    inplace = M[6].clone()
    cum.cum_correct_m4(n, b, inplace, low, M[4], inplace)
    torch.cuda.synchronize()
    check(inplace.cpu().numpy(), ref.cpu().numpy(), tol=1e-11)


def test_supersymmetry_of_diagonal_blocks(cum):
    X = synth.skewed(2000, 8, seed=10)
    C, _ = run(cum, X, 4, 4)
    for d in (3, 4):
        T = blocks.to_dense(C[d], 8, d, 4)
        scale = np.abs(T).max()
        import itertools
        for perm in itertools.permutations(range(d)):
            assert np.abs(np.transpose(T, perm) - T).max() <= 1e-12 * scale


def test_mean_shift_invariance(cum):
    X = synth.skewed(5000, 9, seed=11)
    C0, _ = run(cum, X, 4, 3)
    C1, _ = run(cum, X + np.linspace(-300, 800, 9), 4, 3)
    for d in (2, 3, 4):
        check(C1[d], C0[d], tol=1e-9)


@pytest.mark.parametrize("prec", [0, 2])
def test_rademacher_design_closed_form(cum, prec):
    """The full 2^5-row sign design is exactly 5 independent +-1 variables: every
    mixed cumulant is 0 and the diagonal ones are kappa_d = d! [tau^d] log cosh
    (tests/golden/rademacher_cumulants.json), orders 2..6.  Mixed by an integer
    matrix A, C_d(SA) = C_d(S) x_1 A ... x_d A.  Every intermediate is a small
    dyadic number, so both paths must be exact."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "rademacher_cumulants.json")))["kappa"]
    S = synth.rademacher_design(5)
    A = synth.integer_matrix(5, 6, seed=31)
    for X, n in ((S, 5), (S @ A, 6)):
        C, _ = run(cum, X, 6, 2, prec=prec, dtype="f64" if prec == 0 else "f32")
        for d in range(2, 7):
            ref = np.zeros((5,) * d)
            for i in range(5):
                ref[(i,) * d] = gold[str(d)]
            for _ in range(d if n == 6 else 0):
                ref = np.tensordot(ref, A, axes=([0], [0]))   # mode products, one mode at a time
            got = blocks.to_dense(C[d], n, d, 2)
            assert np.abs(got - ref).max() <= 1e-9 * max(1.0, np.abs(ref).max()), (n, d)


@pytest.mark.parametrize("prec", [0, 2])
def test_power_of_two_column_scaling_is_exact(cum, prec):
    """Scaling column v by 2^k_v scales every cumulant entry by 2^(sum of k over
    its indices), bit for bit: centring, products, FP64 folds, the fp16 parts'
    per-variable scaling and the correction all commute with powers of two."""
    n, b = 9, 3
    X = synth.skewed(3000, n, seed=21)
    k = np.array([-3, 0, 2, 4, -1, 1, 3, -2, 0])
    dtype = "f64" if prec == 0 else "f32"
    Xf = X.astype(np.float32).astype(np.float64) if prec else X
    C0, _ = run(cum, Xf, 4, b, prec=prec, dtype=dtype)
    C1, _ = run(cum, Xf * 2.0 ** k, 4, b, prec=prec, dtype=dtype)
    for d in (2, 3, 4):
        S = 2.0 ** k
        for _ in range(d - 1):
            S = np.multiply.outer(S, 2.0 ** k)
        assert np.array_equal(blocks.to_dense(C1[d], n, d, b), blocks.to_dense(C0[d], n, d, b) * S), d


def _sampled(cum, X, dmax, b, count, seed, dtype="f64", prec=0):
    n = X.shape[1]
    C, _ = run(cum, X, dmax, b, prec=prec, dtype=dtype)
    Xo = X.astype(np.float64)
    _, Xc = oracle.center(Xo)
    out = {}
    for d in range(2, dmax + 1):
        idx = synth.sample_indices(n, d, count, seed=seed + d)
        ref = oracle.cumulant_entries(Xc, idx)
        got = C[d][blocks.entry_offsets(idx, n, b)]
        out[d] = (got, ref)
    return out


def test_paper_scale_sampled(cum):
    """t=1e5, n=60 (Student-t + outliers), b=6, orders 2..4: sampled entries."""
    X = synth.paper_scale()
    for d, (got, ref) in _sampled(cum, X, 4, 6, 1500, seed=20).items():
        check(got, ref)


def test_high_order_fp64_sampled(cum):
    """t=2e5, n=48 (Laplace, orthogonal mix), b=4, orders 2..6 on the FP64 path."""
    X = synth.high_order(dtype=np.float64)
    for d, (got, ref) in _sampled(cum, X, 6, 4, 300, seed=30).items():
        check(got, ref)


def test_device_status_clean(cum):
    import torch
    X = torch.from_numpy(synth.skewed(500, 5, seed=12)).cuda()
    ws = cum.workspace(500, 5, 4, 2, 0)
    cum.cumulants(X, 4, 2, 0, ws=ws)
    assert cum.cum_device_status(ws) == cum.CUM_OK
