"""Pins of the oracle against things other than itself.

Each check ties the oracle to a library routine, a closed form, exact rational
arithmetic or the cumulant generating function of Def. 1.4, so that a dropped
term, a wrong sign, a wrong normalisation or a transposed index fails at least
one of them (``test_planted_mistakes_are_caught`` demonstrates this by planting
such mistakes in the oracle).
"""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _stirling2_eq_n1(d, s):
    # Eq. n1: S(d, sigma) = (1/sigma!) sum_j (-1)^(sigma-j) C(sigma, j) j^d
    return sum((-1) ** (s - j) * math.comb(s, j) * j ** d for j in range(s + 1)) // math.factorial(s)


# ------------------------------------------------------------------ partitions

@pytest.mark.parametrize("d", range(1, 8))
def test_set_partitions_are_all_partitions(d):
    sympy = pytest.importorskip("sympy")
    parts = oracle.set_partitions(d)
    assert len(parts) == int(sympy.bell(d))
    seen = set()
    for zeta in parts:
        flat = sorted(p for B in zeta for p in B)
        assert flat == list(range(d))                       # cover, disjoint
        assert all(list(B) == sorted(B) and B for B in zeta)  # sorted, non-empty
        key = frozenset(frozenset(B) for B in zeta)
        assert key not in seen
        seen.add(key)
    for s in range(1, d + 1):
        count = sum(1 for z in parts if len(z) == s)
        assert count == _stirling2_eq_n1(d, s)
        assert count == int(sympy.functions.combinatorial.numbers.stirling(d, s))


def test_no_singleton_counts_match_paper():
    g = _golden("partition_counts.json")
    sprime = {}
    for d in range(1, 9):
        for zeta in oracle.set_partitions(d):
            if all(len(B) >= 2 for B in zeta):
                sprime[(d, len(zeta))] = sprime.get((d, len(zeta)), 0) + 1
    for d, s, v in g["S_prime"]:
        assert sprime[(d, s)] == v
    F = {d: sum(v for (dd, s), v in sprime.items() if dd == d) for d in range(1, 9)}
    bell = {d: len(oracle.set_partitions(d)) for d in range(1, 9)}
    assert F[1] == g["F_recurrence"]["F1"]
    for d in range(1, 8):
        assert F[d + 1] == bell[d] - F[d]          # Eq. req
    assert [F[d] for d in range(1, 7)] == [0, 1, 1, 4, 11, 41]
    for d, v in g["N"]:
        assert sum((s - 1) * sprime.get((d, s), 0) for s in range(2, d // 2 + 1)) == v


# ------------------------------------------------------------------ library routines

def test_order2_is_biased_covariance():
    X = synth.skewed(500, 6, seed=11)
    C2 = oracle.cumulant_dense(X, 2)
    np.testing.assert_allclose(C2, np.cov(X, rowvar=False, bias=True), rtol=1e-12, atol=1e-13)


def test_diagonals_match_scipy_moments():
    stats = pytest.importorskip("scipy.stats")
    X = synth.skewed(800, 4, seed=12)
    C3 = oracle.cumulant_dense(X, 3)
    C4 = oracle.cumulant_dense(X, 4)
    for i in range(4):
        x = X[:, i]
        np.testing.assert_allclose(C3[i, i, i], stats.moment(x, 3), rtol=1e-11)
        var = np.var(x)
        np.testing.assert_allclose(C4[i, i, i, i], stats.kurtosis(x, fisher=True, bias=True) * var ** 2,
                                   rtol=1e-10)
        np.testing.assert_allclose(C3[i, i, i], stats.skew(x, bias=True) * var ** 1.5, rtol=1e-10)


# ------------------------------------------------------------------ closed forms

def _rademacher_kappa():
    sympy = pytest.importorskip("sympy")
    tau = sympy.Symbol("tau")
    ser = sympy.series(sympy.log(sympy.cosh(tau)), tau, 0, 8).removeO()
    return {d: int(ser.coeff(tau, d) * sympy.factorial(d)) for d in range(2, 7)}


def test_rademacher_kappa_golden():
    g = _golden("rademacher_cumulants.json")["kappa"]
    assert {int(k): v for k, v in g.items()} == _rademacher_kappa()


def _closed_form(A, kappa, d):
    """C_d(S A) for S with independent columns of cumulant kappa_d: multilinearity."""
    k, n = A.shape
    out = np.zeros((n,) * d)
    for a in range(k):
        T = np.array(kappa[d], dtype=np.float64)
        for _ in range(d):
            T = np.multiply.outer(T, A[a])
        out += T
    return out


@pytest.mark.parametrize("d", [2, 3, 4, 5, 6])
def test_rademacher_design_closed_form(d):
    kappa = _rademacher_kappa()
    S = synth.rademacher_design(4)          # t = 16, exactly independent +-1 columns
    A = synth.integer_matrix(4, 3, seed=5)
    X = S @ A
    expect = _closed_form(A, kappa, d)
    dense = oracle.cumulant_dense(X, d)
    scale = max(1.0, np.abs(expect).max())
    np.testing.assert_allclose(dense, expect, rtol=0, atol=1e-12 * scale)
    exact = oracle.cumulant_exact(X, d)
    for idx, v in exact.items():
        assert v == Fraction(int(expect[idx])) and float(expect[idx]).is_integer()
    _, Xc = oracle.center(X)
    idx = np.array(list(itertools.product(range(3), repeat=d)), dtype=np.int32)
    got = oracle.cumulant_entries(Xc, idx)
    np.testing.assert_allclose(got, expect[tuple(idx.T)], rtol=0, atol=1e-12 * scale)


def test_exact_small_integer_data():
    # zero-mean integer data (each row paired with its negation) keeps every
    # intermediate of the FP64 oracle exactly representable
    base = synth.small_integers(8, 3, seed=21, lo=-2, hi=2)
    X = np.vstack([base, -base])
    for d in (2, 3, 4, 5, 6):
        dense = oracle.cumulant_dense(X, d)
        exact = oracle.cumulant_exact(X, d)
        for idx, v in exact.items():
            assert Fraction(dense[idx]) == v, (d, idx)


def test_cgf_definition_sympy():
    """Def. 1.4 with Eq. cum_ge: c_i = d^d K / d tau_i1..d tau_id at 0, K = log((1/t) sum exp(x.tau))."""
    sympy = pytest.importorskip("sympy")
    rows = [[1, 0], [0, 2], [-1, 1], [2, -1], [3, 1]]
    t1, t2 = sympy.symbols("t1 t2")
    taus = [t1, t2]
    K = sympy.log(sum(sympy.exp(r[0] * t1 + r[1] * t2) for r in rows) / len(rows))
    X = np.array(rows, dtype=np.float64)
    for d in (2, 3, 4):
        exact = oracle.cumulant_exact(X, d)
        for idx in itertools.combinations_with_replacement(range(2), d):
            v = sympy.diff(K, *[taus[i] for i in idx]).subs({t1: 0, t2: 0})
            assert sympy.nsimplify(v) == sympy.Rational(exact[idx].numerator, exact[idx].denominator), idx
    # one variable, orders 5 and 6
    tau = sympy.Symbol("tau")
    xs = [1, 0, -1, 2, 3, 3]
    K1 = sympy.log(sum(sympy.exp(x * tau) for x in xs) / len(xs))
    for d in (5, 6):
        exact = oracle.cumulant_exact(np.array(xs, dtype=np.float64)[:, None], d)
        v = sympy.diff(K1, tau, d).subs(tau, 0)
        e = exact[(0,) * d]
        assert sympy.nsimplify(v) == sympy.Rational(e.numerator, e.denominator)


# ------------------------------------------------------------------ invariants

def test_supersymmetry():
    X = synth.skewed(300, 4, seed=31)
    for d in (3, 4, 5):
        C = oracle.cumulant_dense(X, d)
        scale = np.abs(C).max()
        for perm in itertools.permutations(range(d)):
            np.testing.assert_allclose(np.transpose(C, perm), C, rtol=0, atol=1e-13 * scale)


def test_mean_shift_invariance():
    X = synth.skewed(400, 3, seed=41)
    shift = np.array([1e3, -250.0, 7.5])
    for d in (2, 3, 4):
        a = oracle.cumulant_dense(X, d)
        b = oracle.cumulant_dense(X + shift, d)
        np.testing.assert_allclose(b, a, rtol=0, atol=1e-9 * np.abs(a).max())


def test_multilinearity():
    X = synth.skewed(300, 3, seed=51)
    A = np.random.default_rng(52).standard_normal((3, 3))
    for d in (2, 3, 4):
        C = oracle.cumulant_dense(X, d)
        T = C
        for _ in range(d):
            T = np.tensordot(T, A, axes=([0], [0]))   # contract the leading mode with A
        np.testing.assert_allclose(oracle.cumulant_dense(X @ A, d), T, rtol=0, atol=1e-11 * np.abs(T).max())


def test_sample_split_reduction():
    """Alg. 3 / Eq. mapred: the moment of X is the t_s/t weighted sum of the chunk moments."""
    _, Xc = oracle.center(synth.skewed(1003, 3, seed=61))
    cuts = [0, 250, 600, 1003]
    for d in (2, 3, 4):
        full = oracle.moment_dense(Xc, d)
        acc = sum((b - a) / 1003 * oracle.moment_dense(Xc[a:b], d) for a, b in zip(cuts, cuts[1:]))
        np.testing.assert_allclose(acc, full, rtol=1e-12, atol=1e-14)


def test_c_oracle_matches_dense():
    X = synth.skewed(700, 5, seed=71)
    _, Xc = oracle.center(X)
    for d in (2, 3, 4, 5):
        idx = synth.sample_indices(5, d, 60, seed=72 + d)
        dense = oracle.cumulant_dense(X, d)
        np.testing.assert_allclose(oracle.cumulant_entries(Xc, idx), dense[tuple(idx.T)],
                                   rtol=0, atol=1e-12 * np.abs(dense).max())
        mom = oracle.moment_dense(Xc, d)
        np.testing.assert_allclose(oracle.moment_entries(Xc, idx), mom[tuple(idx.T)], rtol=1e-13, atol=1e-15)


def test_gaussian_higher_cumulants_vanish():
    # large-sample check: cumulants of order >= 3 of Gaussian data are 0 up to sampling error
    X = synth.gaussian(200_000, 2, seed=81)
    _, Xc = oracle.center(X)
    for d in (3, 4):
        idx = np.array(list(itertools.product(range(2), repeat=d)), dtype=np.int32)
        c = oracle.cumulant_entries(Xc, idx)
        assert np.abs(c).max() < 0.1


# ------------------------------------------------------------------ planted mistakes

def test_planted_mistakes_are_caught(monkeypatch):
    """Each plausible mistake planted in the oracle fails one of the pins above."""
    kappa = _rademacher_kappa()
    S = synth.rademacher_design(4)
    A = synth.integer_matrix(4, 3, seed=5)
    X = S @ A
    expect4 = _closed_form(A, kappa, 4)
    real_parts = oracle.set_partitions

    # (1) a dropped partition term (a pair partition: singleton terms vanish on centred data)
    def dropped(d):
        p = real_parts(d)
        k = next((i for i, z in enumerate(p) if len(z) > 1 and all(len(B) >= 2 for B in z)), None)
        return p if k is None else p[:k] + p[k + 1:]
    monkeypatch.setattr(oracle, "set_partitions", dropped)
    assert not np.allclose(oracle.cumulant_dense(X, 4), expect4)
    monkeypatch.setattr(oracle, "set_partitions", real_parts)

    # (2) a wrong sign in the (|zeta|-1)! (-1)^(|zeta|-1) coefficient
    class _BadMath:
        def __getattr__(self, k):
            return getattr(math, k)

        @staticmethod
        def factorial(k):
            return -math.factorial(k) if k == 1 else math.factorial(k)
    monkeypatch.setattr(oracle, "math", _BadMath())
    assert not np.allclose(oracle.cumulant_dense(X, 4), expect4)
    monkeypatch.setattr(oracle, "math", math)

    # (3) 1/(t-1) instead of 1/t
    real_moment = oracle.moment_dense
    monkeypatch.setattr(oracle, "moment_dense",
                        lambda Xc, d: real_moment(Xc, d) * Xc.shape[0] / (Xc.shape[0] - 1))
    Y = synth.skewed(50, 3, seed=9)
    assert not np.allclose(oracle.cumulant_dense(Y, 2), np.cov(Y, rowvar=False, bias=True), rtol=1e-6)
    monkeypatch.setattr(oracle, "moment_dense", real_moment)

    # (4) a mis-indexed term: one partition replaced by a copy of another
    def misindexed(d):
        p = real_parts(d)
        pairs = [i for i, z in enumerate(p) if len(z) > 1 and all(len(B) >= 2 for B in z)]
        if len(pairs) < 2:
            return p
        p = list(p)
        p[pairs[0]] = p[pairs[1]]
        return p
    monkeypatch.setattr(oracle, "set_partitions", misindexed)
    assert not np.allclose(oracle.cumulant_dense(X, 4), expect4)
    assert any(v != Fraction(int(expect4[k])) for k, v in oracle.cumulant_exact(X, 4).items())
    monkeypatch.setattr(oracle, "set_partitions", real_parts)
