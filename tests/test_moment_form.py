"""The moment form of the order-6 correction, restated on the oracle's dense
tensors (CPU).

The library's order-6 correction (cum_correct_m4, and cum_cumulants whenever
orders up to 6 are asked for) groups the partitions of Eq. cum_r by the part
that holds the first position.  Where that part is a pair {0, x}, the other four
positions R are one part (C_4[R]) or two pairs (three pairings of C_2 C_2), and
Eq. cum_r at order 4 makes their sum the moment M_4[R].  So

    C_6 = M_6 - sum_x C_2[0x] M_4[R_x] - sum_{pairs P without 0} C_2[P] C_4[rest]
              - sum_{3+3 with 0 in the first triple} C_3 C_3,

25 products instead of the 40 partitions.  These checks tie that identity to the
oracle (moment-to-cumulant formula over all set partitions, Eq. cumfmom), both in
floating point and exactly in rational arithmetic.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

L = "abcdef"


def _term(A, B, FA, FB):
    subs = "".join(L[k] for k in A) + "," + "".join(L[k] for k in B) + "->" + L
    return np.einsum(subs, FA, FB, optimize=False)


def moment_form_c6(M6, M4, C2, C3, C4):
    out = M6.copy()
    nterms = 0
    for x in range(1, 6):                                   # pair {0, x}: C_2 M_4
        out -= _term((0, x), [k for k in range(1, 6) if k != x], C2, M4)
        nterms += 1
    for P in itertools.combinations(range(1, 6), 2):        # pair without 0: C_2 C_4
        out -= _term(P, [k for k in range(6) if k not in P], C2, C4)
        nterms += 1
    for T in itertools.combinations(range(1, 6), 2):        # triples {0} + T: C_3 C_3
        A = (0,) + T
        out -= _term(A, [k for k in range(6) if k not in A], C3, C3)
        nterms += 1
    assert nterms == 25
    return out


@pytest.mark.parametrize("seed", [1, 2])
def test_moment_form_matches_the_oracle(seed):
    X = synth.skewed(400, 4, seed=700 + seed)
    _, Xc = oracle.center(X)
    C = {d: oracle.cumulant_dense(X, d) for d in (2, 3, 4, 6)}
    got = moment_form_c6(oracle.moment_dense(Xc, 6), oracle.moment_dense(Xc, 4), C[2], C[3], C[4])
    err = np.abs(got - C[6]).max() / np.abs(C[6]).max()
    assert err < 1e-12, err


def test_moment_form_is_exact_on_integer_data():
    """Exact rational arithmetic on small integer data (n = 2, every entry)."""
    X = synth.small_integers(16, 2, seed=9)
    t, n = X.shape
    rows = [[Fraction(int(v)) for v in r] for r in X]
    mean = [sum(r[i] for r in rows) / t for i in range(n)]
    xc = [[r[i] - mean[i] for i in range(n)] for r in rows]

    def moment(idx):
        s = Fraction(0)
        for r in xc:
            p = Fraction(1)
            for i in idx:
                p *= r[i]
            s += p
        return s / t

    def cum(idx):
        # Eq. cumfmom over all set partitions of the positions of idx
        tot = Fraction(0)
        for zeta in oracle.set_partitions(len(idx)):
            s = len(zeta)
            p = Fraction((-1) ** (s - 1) * math.factorial(s - 1))
            for B in zeta:
                p *= moment([idx[k] for k in B])
            tot += p
        return tot

    for idx in itertools.product(range(n), repeat=6):
        rhs = moment(idx)
        for x in range(1, 6):
            R = [idx[k] for k in range(1, 6) if k != x]
            rhs -= cum([idx[0], idx[x]]) * moment(R)
        for P in itertools.combinations(range(1, 6), 2):
            rhs -= cum([idx[k] for k in P]) * cum([idx[k] for k in range(6) if k not in P])
        for T in itertools.combinations(range(1, 6), 2):
            A = (0,) + T
            rhs -= cum([idx[k] for k in A]) * cum([idx[k] for k in range(6) if k not in A])
        assert rhs == cum(list(idx)), idx
