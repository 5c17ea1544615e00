"""Seeded synthetic inputs shared by the oracle tests, the GPU parity tests and bench.py.

This module holds data generation only: it computes no moment, cumulant,
centring or block-structure quantity.  Every generator is deterministic in its
seed (numpy ``default_rng``).

The five workload recipes stand in for the paper's unspecified "illustrative
data" (Sec. 5.2.2) and mirror the scales of its block-size and multiprocessing
runs (n = 60, t = 2e5; Sec. 5.2.1 and 5.2.3).  Each adds per-column offsets
U(-5, 5) so that centring (Def. 1.3) is exercised.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 170105420


@dataclass(frozen=True)
class Workload:
    """One workload: data shape, the orders computed and the block side b."""
    name: str
    t: int
    n: int
    b: int
    d_max: int
    dtype: str            # "f64" or "f32": element type of X as handed to the library
    seed: int
    orders: tuple = field(default=(2, 3, 4))


WORKLOADS = {
    "paper-small": Workload("paper-small", 2000, 20, 4, 4, "f64", BASE_SEED + 1, (2, 3, 4)),
    "paper-scale": Workload("paper-scale", 100_000, 60, 6, 4, "f64", BASE_SEED + 2, (2, 3, 4)),
    "precision": Workload("precision", 1_000_000, 128, 16, 3, "f32", BASE_SEED + 3, (2, 3)),
    "high-order": Workload("high-order", 200_000, 48, 4, 6, "f32", BASE_SEED + 4, (2, 3, 4, 5, 6)),
}


def _offsets(rng, n):
    return rng.uniform(-5.0, 5.0, size=n)


def student_t_mixed(t, n, seed, nu=5.0, mix="uniform"):
    """Student-t(nu) columns mixed by a seeded n x n matrix plus column offsets."""
    rng = np.random.default_rng(seed)
    S = rng.standard_t(nu, size=(t, n))
    if mix == "uniform":
        A = rng.uniform(-1.0, 1.0, size=(n, n))
    else:
        A = rng.standard_normal((n, n))
    return S @ A + _offsets(rng, n)


def paper_small(seed=BASE_SEED + 1, t=2000, n=20):
    """t x n float64, Student-t(5) columns mixed by U(-1,1) n x n."""
    return student_t_mixed(t, n, seed, nu=5.0, mix="uniform")


def paper_scale(seed=BASE_SEED + 2, t=100_000, n=60, outlier_frac=0.05):
    """t x n float64, Student-t(4) mixed by N(0,1) n x n; 5% of rows replaced by 3*N(0,I)."""
    rng = np.random.default_rng(seed)
    S = rng.standard_t(4.0, size=(t, n))
    A = rng.standard_normal((n, n))
    X = S @ A
    k = int(round(outlier_frac * t))
    rows = rng.choice(t, size=k, replace=False)
    X[rows] = 3.0 * rng.standard_normal((k, n))
    return X + _offsets(rng, n)


def _skewnorm_quantile(alpha, lo=-8.0, hi=10.0, points=2_000_001):
    """Quantile function of the skew-normal(alpha) law as a monotone table: its
    density 2 phi(x) Phi(alpha x) integrated by the trapezoid rule on a fine
    grid, inverted by linear interpolation."""
    from scipy import special
    x = np.linspace(lo, hi, points)
    pdf = 2.0 * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi) * special.ndtr(alpha * x)
    F = np.concatenate([[0.0], np.cumsum(0.5 * (pdf[1:] + pdf[:-1]) * np.diff(x))])
    F /= F[-1]
    keep = np.concatenate([[True], np.diff(F) > 0])
    return F[keep], x[keep]


def precision(seed=BASE_SEED + 3, t=1_000_000, n=128, rho=0.6, alpha=4.0, chunk=131072):
    """t x n float32: skew-normal(alpha) marginals under a Gaussian copula, AR(1) rho."""
    from scipy import special
    rng = np.random.default_rng(seed)
    idx = np.arange(n)
    Sigma = rho ** np.abs(idx[:, None] - idx[None, :])
    L = np.linalg.cholesky(Sigma)
    off = _offsets(rng, n)
    Fq, xq = _skewnorm_quantile(alpha)
    out = np.empty((t, n), dtype=np.float32)
    for s in range(0, t, chunk):
        e = min(t, s + chunk)
        G = rng.standard_normal((e - s, n))
        U = special.ndtr(G @ L.T)
        out[s:e] = (np.interp(U, Fq, xq) + off).astype(np.float32)
    return out


def _orthogonal(rng, n):
    Q, R = np.linalg.qr(rng.standard_normal((n, n)))
    return Q * np.sign(np.diag(R))[None, :]


def high_order(seed=BASE_SEED + 4, t=200_000, n=48, dtype=np.float32):
    """t x n: Laplace marginals mixed by a seeded orthogonal n x n matrix."""
    rng = np.random.default_rng(seed)
    S = rng.laplace(size=(t, n))
    Q = _orthogonal(rng, n)
    return (S @ Q + _offsets(rng, n)).astype(dtype)


def batch_specs(seed=BASE_SEED + 5, count=512, t_lo=5000, t_hi=200_000, ns=(16, 32, 48, 64, 96)):
    """(t, n, seed) for each dataset of the batched workload: t log-uniform, n uniform."""
    rng = np.random.default_rng(seed)
    ts = np.rint(np.exp(rng.uniform(math.log(t_lo), math.log(t_hi), size=count))).astype(np.int64)
    nn = rng.choice(np.asarray(ns), size=count)
    seeds = rng.integers(0, 2**31 - 1, size=count)
    return [(int(a), int(b), int(c)) for a, b, c in zip(ts, nn, seeds)]


def batch_dataset(t, n, seed):
    """One dataset of the batched workload: float32 Student-t(5) mixed by U(-1,1)."""
    return student_t_mixed(t, n, seed, nu=5.0, mix="uniform").astype(np.float32)


def make(name, dtype=None):
    """Data for a named workload."""
    if name == "paper-small":
        X = paper_small()
    elif name == "paper-scale":
        X = paper_scale()
    elif name == "precision":
        X = precision()
    elif name == "high-order":
        X = high_order(dtype=np.float64 if dtype == "f64" else np.float32)
    else:
        raise KeyError(name)
    return X


# ---- small structured inputs for tests -------------------------------------------------

def gaussian(t, n, seed, offset=True):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((t, n))
    if offset:
        X = X + _offsets(rng, n)
    return X


def skewed(t, n, seed):
    """Exponential columns mixed by U(-1,1): non-zero odd cumulants at every order."""
    rng = np.random.default_rng(seed)
    S = rng.exponential(size=(t, n))
    A = rng.uniform(-1.0, 1.0, size=(n, n))
    return S @ A + _offsets(rng, n)


def small_integers(t, n, seed, lo=-3, hi=3):
    """Integer-valued float64 data (exactly representable)."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=(t, n)).astype(np.float64)


def rademacher_design(k):
    """All 2**k sign patterns of k +-1 variables (rows), as float64.

    The empirical distribution of these rows is exactly k independent
    symmetric +-1 variables."""
    t = 1 << k
    rows = np.arange(t)[:, None]
    bits = (rows >> np.arange(k)[None, :]) & 1
    return (2.0 * bits - 1.0).astype(np.float64)


def integer_matrix(k, n, seed, lo=-2, hi=2):
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=(k, n)).astype(np.float64)


def sample_indices(n, d, count, seed, include_special=True):
    """Seeded multi-indices in [0, n)^d, including all-equal and repeated patterns."""
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, n, size=(count, d))
    if include_special and count >= 8:
        special = []
        for v in (0, n - 1, n // 2):
            special.append([v] * d)
        special.append([0] * (d - 1) + [n - 1])
        special.append(list(range(min(d, n))) + [0] * (d - min(d, n)))
        special.append([n - 1] * (d // 2) + [0] * (d - d // 2))
        special = np.asarray(special[: count], dtype=np.int64)
        idx[: len(special)] = special
    return idx.astype(np.int32)
