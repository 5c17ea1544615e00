"""Failure detection without a GPU fault: every wait of the contraction kernels
is bounded, and an expired wait is reported through the workspace status word
instead of hanging.  cum_probe_bounded_wait runs that same wait on a barrier
nothing arrives at; the host must read CUM_ETIMEOUT, and the device must stay
usable afterwards."""
import time

import numpy as np
import pytest

import blocks
import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cum():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1701_05420_gb300 as m
    return m


def test_expired_wait_is_reported_and_device_stays_usable(cum):
    import torch
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
    assert cum.cum_device_status(ws) == cum.CUM_OK
    t0 = time.perf_counter()
    cum.cum_probe_bounded_wait(ws)
    status = cum.cum_device_status(ws)          # synchronises the stream
    elapsed = time.perf_counter() - t0
    assert status == cum.CUM_ETIMEOUT
    assert elapsed < 60.0
    assert cum.cum_device_status(ws) == cum.CUM_OK   # reading cleared it
    # a full computation on the same device afterwards
    X = synth.skewed(2000, 9, seed=77)
    C, _ = cum.cumulants(torch.from_numpy(X).cuda(), 4, 3, cum.CUM_PREC_FP16X3)
    torch.cuda.synchronize()
    for d in (2, 3, 4):
        relF, _ = blocks.rel_errors(blocks.to_dense(C[d].cpu().numpy(), 9, d, 3), oracle.cumulant_dense(X, d))
        assert relF <= 1e-6, (d, relF)


def test_probe_rejects_bad_workspace(cum):
    import torch
    with pytest.raises(cum.CumError):
        cum.cum_probe_bounded_wait(torch.zeros(16, dtype=torch.uint8, device="cuda"))
