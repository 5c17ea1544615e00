"""Test-side reading of the block storage documented in include/cumgb.h.

Written independently of the library: block ranks come from sorting all
sorted tuples in colex order (compare reversed tuples), not from the
combinatorial-number-system formula the library uses."""
import functools
import itertools

import numpy as np


@functools.lru_cache(maxsize=None)
def colex_tuples(nbar, d):
    tuples = list(itertools.combinations_with_replacement(range(nbar), d))
    tuples.sort(key=lambda tup: tup[::-1])
    return tuples


@functools.lru_cache(maxsize=None)
def rank_table(nbar, d):
    return {tup: r for r, tup in enumerate(colex_tuples(nbar, d))}


def entry_offsets(idx, n, b):
    """Storage offsets of multi-indices idx (count x d, variable indices < n)."""
    idx = np.asarray(idx)
    count, d = idx.shape
    nbar = -(-n // b)
    table = rank_table(nbar, d)
    blk = idx // b
    inb = idx % b
    perm = np.argsort(blk, axis=1, kind="stable")
    js = np.take_along_axis(blk, perm, axis=1)
    iis = np.take_along_axis(inb, perm, axis=1)
    w = b ** np.arange(d - 1, -1, -1)
    ranks = np.array([table[tuple(r)] for r in js.tolist()], dtype=np.int64)
    return ranks * b ** d + (iis * w).sum(axis=1)


def to_dense(C, n, d, b):
    """Expand a block-stored order-d tensor to the full n^d array."""
    C = np.asarray(C)
    nbar = -(-n // b)
    npad = nbar * b
    out = np.zeros((npad,) * d)
    bd = b ** d
    for r, j in enumerate(colex_tuples(nbar, d)):
        blk = C[r * bd:(r + 1) * bd].reshape((b,) * d)
        sl = tuple(slice(jj * b, (jj + 1) * b) for jj in j)
        for perm in set(itertools.permutations(range(d))):
            # place the block at every permutation of its block index
            jp = tuple(j[p] for p in perm)
            slp = tuple(slice(jj * b, (jj + 1) * b) for jj in jp)
            out[slp] = np.transpose(blk, perm)
        del sl
    return out[(slice(0, n),) * d]


def from_dense(T, n, d, b):
    """Block storage of a full n^d super-symmetric tensor (inverse of to_dense)."""
    nbar = -(-n // b)
    npad = nbar * b
    P = np.zeros((npad,) * d)
    P[(slice(0, n),) * d] = T
    bd = b ** d
    out = np.zeros(len(colex_tuples(nbar, d)) * bd)
    for r, j in enumerate(colex_tuples(nbar, d)):
        sl = tuple(slice(jj * b, (jj + 1) * b) for jj in j)
        out[r * bd:(r + 1) * bd] = P[sl].reshape(-1)
    return out


def rel_errors(got, ref):
    """(relF, relMax): normwise relative errors over the compared entries."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    diff = got - ref
    nf = np.linalg.norm(ref)
    nm = np.abs(ref).max()
    return (np.linalg.norm(diff) / nf if nf > 0 else np.linalg.norm(diff),
            np.abs(diff).max() / nm if nm > 0 else np.abs(diff).max())
