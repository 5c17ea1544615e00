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
