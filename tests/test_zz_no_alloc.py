"""cum_cumulants_noalloc: the entry point for callers that cannot allocate device
memory (and so cannot pass a workspace) must give the same cumulant tensors as
cum_cumulants with a caller workspace, call after call, although every call
reuses the library's one fixed device array.

Named to be collected last: a run that stops at the first failure has run
every other test before this one."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 2: 1e-6, 3: 1e-6}   # the parity tolerances of the FP64, FP16x3 and TF32x3 paths


@pytest.fixture(scope="module")
def cum():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1701_05420_gb300 as m
    return m


def _reference(cum, X, d_max, b, prec):
    C, mean = cum.cumulants(X, d_max, b, prec)     # cum_cumulants with a torch-allocated workspace
    return C, mean


def _noalloc(cum, X, d_max, b, prec):
    """Direct C-ABI call of cum_cumulants_noalloc (outputs allocated by the caller)."""
    import torch
    t, n = X.shape
    C = [torch.full((cum.num_entries(n, d, b),), float("nan"), dtype=torch.float64, device=X.device)
         for d in range(2, d_max + 1)]
    mean = torch.full((n,), float("nan"), dtype=torch.float64, device=X.device)
    arr = (ctypes.c_void_p * len(C))(*[c.data_ptr() for c in C])
    dt = cum.CUM_F64 if X.dtype == torch.float64 else cum.CUM_F32
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = cum.lib.cum_cumulants_noalloc(ctypes.c_void_p(X.data_ptr()), dt, t, n, X.stride(0), d_max, b, prec, arr,
                                       ctypes.c_void_p(mean.data_ptr()), stream)
    assert rc == cum.CUM_OK, cum.cum_strerror(rc)
    return {d: C[d - 2] for d in range(2, d_max + 1)}, mean


def _compare(got, ref, tol):
    for d in ref:
        g = got[d].cpu().numpy()
        r = ref[d].cpu().numpy()
        assert np.all(np.isfinite(g)), d
        err = np.linalg.norm(g - r) / max(np.linalg.norm(r), 1e-300)
        assert err <= tol, (d, err)


@pytest.mark.parametrize("prec", [0, 2, 3])
def test_noalloc_matches_workspace_entry_point_twice(cum, prec):
    import torch
    dtype = np.float64 if prec == 0 else np.float32
    # two calls in a row with different data and sizes: the second call must not
    # see anything the first left in the shared array
    cases = [(6000, 13, 3, 5, 401), (2500, 9, 2, 6, 402)]
    for t, n, b, d_max, seed in cases:
        X = torch.from_numpy(synth.skewed(t, n, seed=seed).astype(dtype)).cuda()
        got, gmean = _noalloc(cum, X, d_max, b, prec)
        ref, rmean = _reference(cum, X, d_max, b, prec)
        torch.cuda.synchronize()
        _compare(got, ref, TOL[prec])
        np.testing.assert_allclose(gmean.cpu().numpy(), rmean.cpu().numpy(), rtol=1e-14, atol=1e-14)


def test_noalloc_rejects_requests_beyond_its_array(cum):
    import torch
    t, n, b, d_max = 2_000_000, 48, 4, 6
    assert cum.cum_workspace_size(t, n, d_max, b, 0) > cum.CUM_NOALLOC_WORKSPACE_BYTES
    X = torch.empty((1, n), dtype=torch.float64, device="cuda")   # never read: rejected before any launch
    C = [torch.empty(1, dtype=torch.float64, device="cuda") for _ in range(2, d_max + 1)]
    arr = (ctypes.c_void_p * len(C))(*[c.data_ptr() for c in C])
    rc = cum.lib.cum_cumulants_noalloc(ctypes.c_void_p(X.data_ptr()), cum.CUM_F64, t, n, n, d_max, b, 0, arr, None,
                                       None)
    assert rc == cum.CUM_EUNSUPPORTED
    # an invalid argument is reported as such even when the request is also too large
    arr[1] = None
    rc = cum.lib.cum_cumulants_noalloc(ctypes.c_void_p(X.data_ptr()), cum.CUM_F64, t, n, n, d_max, b, 0, arr, None,
                                       None)
    assert rc == cum.CUM_EINVAL
