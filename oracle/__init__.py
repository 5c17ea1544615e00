"""Reference oracle for moment and cumulant tensors -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import or execute anything in this package.  The library in
``paper_1701_05420_gb300`` never calls it and shares no code with it.

What it computes, written from the paper's definitions (Domino, Gawron, Pawela,
"Efficient computation of higher order cumulant tensors"):

* centring: X~ = X - E(X), per column (Def. 1.3), two-pass in FP64;
* moments:  m_i = (1/t) sum_l prod_k x~_{l,i_k} over the FULL n^d index set,
  symmetry not used (Def. 1.2, Eq. d::moment);
* cumulants: the moment-to-cumulant formula over ALL set partitions of 1:d
  (Eq. cumfmom, Sec. 5.3):
      c_i = sum_zeta (|zeta|-1)! (-1)^(|zeta|-1) prod_{B in zeta} m_{i_B},
  using moments of the centred data of every order 1..d.  This is deliberately
  NOT the recursion the library implements (Eq. cum_r, Alg. 4-5); the two are
  equal by Eq. cum and its proof in App. B.

Three implementations of the same definitions:

* ``moment_dense`` / ``cumulant_dense``: numpy, full n^d tensors (small n);
* ``cumulant_entries``: plain C (``ls_entries.c``), one entry at a time from
  the 2^d - 1 subset moments of that entry -- used for sampled entries of large
  workloads;
* ``cumulant_exact``: pure-Python ``fractions.Fraction`` for tiny integer data.

Readings taken where the paper is silent or garbled: normalisation is 1/t
(Eq. d::moment), not 1/(t-1); "non-crossing" sub-tuples in Def. 3.1 are read as
all set partitions (the Stirling count of Eq. n1 and the c13*c24 term of Eq. c4
require it).

Every function here is pinned by ``tests/test_oracle_pins.py`` against library
routines, closed forms and exact rational arithmetic.
"""
from __future__ import annotations

import ctypes
import math
import os
from fractions import Fraction
from itertools import product as _iproduct

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBNAME = os.path.join(_HERE, "_libls_entries.so")


# ---------------------------------------------------------------- combinatorics

def set_partitions(d):
    """All set partitions of {0, ..., d-1}, as lists of sorted blocks.

    Enumerated by restricted growth strings a_0..a_{d-1} (a_0 = 0,
    a_k <= 1 + max(a_0..a_{k-1})); element k goes to block a_k.  Their number is
    the Bell number B(d); those with sigma blocks number S(d, sigma) (Eq. n1).
    """
    if d == 0:
        return [[]]
    out = []

    def rec(k, a, m):
        if k == d:
            blocks = [[] for _ in range(m + 1)]
            for pos, lab in enumerate(a):
                blocks[lab].append(pos)
            out.append(blocks)
            return
        for lab in range(m + 2):
            a.append(lab)
            rec(k + 1, a, max(m, lab))
            a.pop()

    rec(1, [0], 0)
    return out


# ---------------------------------------------------------------- centring / moments

def center(X):
    """Def. 1.3: X~ = X - E(X), columnwise, in FP64 (two passes: mean, then a
    correction by the mean of the residual)."""
    X = np.asarray(X, dtype=np.float64)
    t = X.shape[0]
    mu = X.sum(axis=0) / t
    R = X - mu
    mu = mu + R.sum(axis=0) / t
    return mu, X - mu


_LETTERS = "abcdefghijklmnopqrstuvwxyz"


def moment_dense(Xc, d):
    """Def. 1.2 / Eq. d::moment: m_i = (1/t) sum_l prod_{k=1..d} x_{l, i_k}
    for every i in [0, n)^d (the full tensor, symmetry not used)."""
    Xc = np.asarray(Xc, dtype=np.float64)
    t = Xc.shape[0]
    if d == 0:
        return np.float64(1.0)
    subs = ",".join("z" + _LETTERS[k] for k in range(d)) + "->" + _LETTERS[:d]
    return np.einsum(subs, *([Xc] * d), optimize=False) / t


def cumulant_dense(X, d, centred=False):
    """Eq. cumfmom: the d-th cumulant tensor (full n^d) from the moments of the
    centred data of orders 1..d, summed over all set partitions of 1:d."""
    Xc = np.asarray(X, dtype=np.float64) if centred else center(X)[1]
    if d == 1:
        return Xc.sum(axis=0) / Xc.shape[0]
    moments = {k: moment_dense(Xc, k) for k in range(1, d + 1)}
    n = Xc.shape[1]
    C = np.zeros((n,) * d)
    for zeta in set_partitions(d):
        s = len(zeta)
        coef = math.factorial(s - 1) * (-1) ** (s - 1)
        subs = ",".join("".join(_LETTERS[p] for p in B) for B in zeta) + "->" + _LETTERS[:d]
        C += coef * np.einsum(subs, *[moments[len(B)] for B in zeta], optimize=False)
    return C


# ---------------------------------------------------------------- sampled entries (plain C)

def _load_c():
    if not os.path.exists(_LIBNAME):
        build_c()
    lib = ctypes.CDLL(_LIBNAME)
    lib.oracle_cumulant_entries.restype = ctypes.c_int
    lib.oracle_cumulant_entries.argtypes = [
        ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int64, ctypes.c_int,
        ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    lib.oracle_moment_entries.restype = ctypes.c_int
    lib.oracle_moment_entries.argtypes = lib.oracle_cumulant_entries.argtypes
    return lib


def build_c(force=False):
    """Compile ls_entries.c with the host C compiler (gcc, OpenMP)."""
    src = os.path.join(_HERE, "ls_entries.c")
    if os.path.exists(_LIBNAME) and not force and os.path.getmtime(_LIBNAME) >= os.path.getmtime(src):
        return _LIBNAME
    import subprocess
    tmp = _LIBNAME + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src, "-lm"], check=True)
    os.replace(tmp, _LIBNAME)
    return _LIBNAME


_lib = None


def _c():
    global _lib
    if _lib is None:
        _lib = _load_c()
    return _lib


def _entries(fn, Xc, idx, threads):
    Xc = np.ascontiguousarray(Xc, dtype=np.float64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    t, n = Xc.shape
    count, d = idx.shape
    out = np.empty(count, dtype=np.float64)
    rc = fn(Xc.ctypes.data, t, n, n, d, count, idx.ctypes.data, out.ctypes.data, int(threads))
    if rc != 0:
        raise ValueError(f"oracle C routine failed with code {rc}")
    return out


def cumulant_entries(Xc, idx, threads=0):
    """Eq. cumfmom for the listed multi-indices idx (count x d) of centred data Xc."""
    return _entries(_c().oracle_cumulant_entries, Xc, idx, threads)


def moment_entries(Xc, idx, threads=0):
    """Eq. d::moment for the listed multi-indices idx (count x d) of centred data Xc."""
    return _entries(_c().oracle_moment_entries, Xc, idx, threads)


# ---------------------------------------------------------------- exact rational oracle

def cumulant_exact(X, d):
    """Eq. cumfmom in exact rational arithmetic (fractions.Fraction), full n^d
    tensor as a dict {multi-index tuple: Fraction}.  Pure Python: tiny inputs
    only (t <= 64, n <= 4, d <= 6).  X may hold ints, Fractions or floats
    (floats are converted exactly)."""
    rows = [[Fraction(v) for v in row] for row in np.asarray(X, dtype=object).tolist()]
    t = len(rows)
    n = len(rows[0])
    mean = [sum(r[i] for r in rows) / t for i in range(n)]
    xc = [[r[i] - mean[i] for i in range(n)] for r in rows]
    memo = {}

    def m(sub):
        key = tuple(sorted(sub))
        if key not in memo:
            s = Fraction(0)
            for r in xc:
                p = Fraction(1)
                for i in key:
                    p *= r[i]
                s += p
            memo[key] = s / t
        return memo[key]

    parts = set_partitions(d)
    out = {}
    for idx in _iproduct(range(n), repeat=d):
        c = Fraction(0)
        for zeta in parts:
            s = len(zeta)
            term = Fraction(math.factorial(s - 1) * (-1) ** (s - 1))
            for B in zeta:
                term *= m([idx[p] for p in B])
            c += term
        out[idx] = c
    return out
