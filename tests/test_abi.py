"""CPU checks of the C ABI: the library loads, exports every declared entry
point, and its host-only functions follow the documented block layout."""
import itertools
import math
import os
import re

import pytest

import blocks

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(cum_[a-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def cum():
    import paper_1701_05420_gb300 as m
    return m


def test_exports_every_declared_symbol(cum):
    names = _declared()
    assert {"cum_center", "cum_moment_blocks", "cum_cumulants", "cum_block_rank", "cum_block_unrank"} <= names
    for name in names:
        assert hasattr(cum.lib, name), name


@pytest.mark.parametrize("nbar,d", [(1, 1), (3, 2), (12, 6), (17, 4), (8, 3), (5, 5)])
def test_num_blocks_is_multiset_count(cum, nbar, d):
    assert cum.cum_num_blocks(nbar, d) == math.comb(nbar + d - 1, d)
    assert cum.cum_num_blocks(nbar, d) == len(blocks.colex_tuples(nbar, d))


def test_high_order_block_count_example(cum):
    # 48 variables in blocks of 4: 12376 order-6 blocks
    assert cum.cum_num_blocks(12, 6) == 12376


@pytest.mark.parametrize("nbar,d", [(1, 3), (4, 2), (6, 4), (12, 3), (7, 6)])
def test_rank_unrank_roundtrip(cum, nbar, d):
    for r, tup in enumerate(blocks.colex_tuples(nbar, d)):
        assert cum.cum_block_rank(list(tup)) == r
        assert cum.cum_block_unrank(r, d, nbar) == list(tup)


def test_rank_rejects_bad_tuples(cum):
    with pytest.raises(cum.CumError):
        cum.cum_block_rank([2, 1])
    with pytest.raises(cum.CumError):
        cum.cum_block_rank([-1, 0])
    with pytest.raises(cum.CumError):
        cum.cum_block_unrank(10, 2, 3)   # only 6 blocks


def test_workspace_size(cum):
    for prec in (cum.CUM_PREC_FP64, cum.CUM_PREC_BF16X3, cum.CUM_PREC_FP16X3, cum.CUM_PREC_TF32X3):
        s2 = cum.cum_workspace_size(2000, 20, 2, 4, prec)
        s4 = cum.cum_workspace_size(2000, 20, 4, 4, prec)
        assert 0 < s2 <= s4
    assert cum.cum_workspace_size(0, 20, 4, 4, 0) == 0
    assert cum.cum_workspace_size(100, 20, 7, 4, 0) == 0      # order above the supported maximum
    assert cum.cum_workspace_size(100, 20, 4, 4, 4) == 0      # unknown precision
    assert cum.cum_workspace_size(100, 300, 3, 4, cum.CUM_PREC_BF16X3) == 0   # too many variables to stage


def test_argument_errors_without_gpu(cum):
    lib = cum.lib
    assert lib.cum_center(None, 0, 10, 3, 3, 1, 0, None, None, 0, None) == cum.CUM_EINVAL
    assert lib.cum_moment_blocks(1, 10, 3, 1, 0, None, None, 0, None) == cum.CUM_EINVAL
    assert lib.cum_cumulants(None, 0, 10, 3, 3, 4, 1, 0, None, None, None, 0, None) == cum.CUM_EINVAL
    assert lib.cum_correct(7, 3, 1, None, None, None, None) == cum.CUM_EINVAL
    assert cum.cum_strerror(cum.CUM_ETIMEOUT)
    assert cum.cum_strerror(99) == "unknown status"


def test_workspace_too_small_is_reported(cum):
    import ctypes
    buf = ctypes.create_string_buffer(1024 + 256)
    addr = (ctypes.addressof(buf) + 255) // 256 * 256
    fake_x = ctypes.c_void_p(addr)
    rc = cum.lib.cum_center(fake_x, 1, 1000, 4, 4, 2, 0, None, ctypes.c_void_p(addr), 1024, None)
    assert rc == cum.CUM_EWORKSPACE


def _tc_cost(tiles, steps, S, ctas=152, unit_steps=24):
    per = -(-steps // S)
    return -(-tiles * S // ctas) * (per + unit_steps)


def _tiles(t, n, b, d, tile_m, tile_n):
    """Active tiles of the staircase contraction for tile_m x tile_n tiles:
    row tile I starts at a row whose last block index is c; its valid columns
    are the leading C(nbar - c + dB - 1, dB) b^dB ones.  Counted here from
    explicit tuple lists, independently of the library's closed form."""
    import itertools
    nbar = -(-n // b)
    dA, dB = (d + 1) // 2, d // 2
    rows = sorted(itertools.combinations_with_replacement(range(nbar), dA), key=lambda u: u[::-1])
    cols = list(itertools.combinations_with_replacement(range(nbar), dB))
    lasts = [u[-1] for u in rows for _ in range(b ** dA)]
    total = 0
    for r0 in range(0, len(lasts), tile_m):
        c = lasts[r0]
        ncols = sum(b ** dB for u in cols if u[0] >= c)
        total += -(-ncols // tile_n)
    return total


@pytest.mark.parametrize("prec,tile_m,tile_n,workers", [(3, 256, 128, 76), (2, 256, 128, 76), (1, 256, 128, 76)])
@pytest.mark.parametrize("t,n,b,d", [
    (200_000, 48, 4, 2), (200_000, 48, 4, 3), (200_000, 48, 4, 4), (200_000, 48, 4, 5), (200_000, 48, 4, 6),
    (100_000, 60, 6, 3), (100_000, 60, 6, 4), (1_000_000, 128, 16, 2), (1_000_000, 128, 16, 3),
    (9000, 20, 4, 4), (2000, 20, 4, 4), (77_777, 96, 8, 4),
])
def test_tc_split_minimises_the_busiest_worker(cum, t, n, b, d, prec, tile_m, tile_n, workers):
    """The tensor-core t-axis split (Alg. 3) takes the S that minimises the
    busiest worker's time under round-robin units: ceil(units / workers) units
    of (chunk steps + 24) 128-sample steps each; the smallest S on a tie.
    Outside batches every split precision runs CTA pairs on 256 x 128 tiles
    (76 workers)."""
    p = cum.cum_plan_info(d, t, n, b, prec)
    assert p["tile_m"] == tile_m and p["tile_n"] == tile_n
    if d <= 4 and n <= 60:
        assert p["active_tiles"] == _tiles(t, n, b, d, tile_m, tile_n)
    t_pad = -(-t // 128) * 128
    steps = t_pad // 128
    S = p["splits"]
    assert p["units"] == p["active_tiles"] * S
    assert p["chunk"] % 128 == 0 and p["chunk"] * S >= t_pad > p["chunk"] * (S - 1)
    smax = max(1, min(t_pad // 2048, (1 << 30) // (8 * cum.num_entries(n, d, b)), 1024))
    costs = {s: _tc_cost(p["active_tiles"], steps, s, ctas=workers) for s in range(1, smax + 1)
             if -(-steps // -(-steps // s)) == s}
    best = min(costs.values())
    assert _tc_cost(p["active_tiles"], steps, S, ctas=workers) == best
    assert S == min(s for s, c in costs.items() if c == best)


def test_tc_split_of_the_high_order_workload(cum):
    # the CTA-pair plans of the high-order workload, orders 2..6 (every split precision)
    for prec in (cum.CUM_PREC_BF16X3, cum.CUM_PREC_FP16X3, cum.CUM_PREC_TF32X3):
        got = [cum.cum_plan_info(d, 200_000, 48, 4, prec)["splits"] for d in range(2, 7)]
        assert got == [75, 15, 4, 2, 2]


def test_fp64_split_fills_eight_units_per_sm(cum):
    for (t, n, b, d) in [(200_000, 48, 4, 4), (100_000, 60, 6, 3), (9000, 20, 4, 4)]:
        p = cum.cum_plan_info(d, t, n, b, cum.CUM_PREC_FP64)
        t_pad = -(-t // 128) * 128
        smax = max(1, min(t_pad // 1024, (1 << 30) // (8 * cum.num_entries(n, d, b)), 1024))
        S = min(-(-8 * 160 // p["active_tiles"]), smax)
        per = -(-(t_pad // 16) // S)
        assert p["chunk"] == per * 16 and p["splits"] == -(-(t_pad // 16) // per)


def test_batch_splits_only_to_balance_the_pool(cum):
    """In a batch every dataset's units share the CTAs: a dataset is split only
    until its units are within an eighth of a CTA's average work."""
    specs = [(5000 + 3000 * i, (16, 32, 48)[i % 3]) for i in range(40)]
    ts, ns = [t for t, _ in specs], [n for _, n in specs]
    d_max, b, prec = 4, 4, cum.CUM_PREC_FP16X3
    B = cum.Batch(ts, ns, [b] * len(specs), d_max, prec)
    try:
        units = B.info()["units"]
    finally:
        B.close()
    expect = 0
    for d in range(2, d_max + 1):
        # the batch runs the one-CTA kernel on 128 x 128 tiles at every order
        tiles = [_tiles(t, n, b, d, 128, 128) for t, n in specs]
        steps = [-(-t // 128) for t in ts]
        work = sum(a * (s + 24) for a, s in zip(tiles, steps))
        cap = max(16, -(-work // (8 * 152)))
        for a, s, t, n in zip(tiles, steps, ts, ns):
            smax = max(1, min(s * 128 // 2048, (1 << 30) // (8 * cum.num_entries(n, d, b)), 1024))
            S = min(-(-s // cap), smax)
            per = -(-s // S)
            expect += a * -(-s // per)
    assert units == expect
    single = sum(cum.cum_plan_info(d, t, n, b, cum.CUM_PREC_TF32X3)["units"] for t, n in specs
                 for d in range(2, d_max + 1))
    assert units < single
