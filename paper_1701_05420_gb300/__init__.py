"""Block-structured moment and cumulant tensors on GB300 (sm_103a).

Thin Python binding of the C ABI in ``include/cumgb.h`` (library
``_lib/libcumgb.so``, built in-tree by ``build.py``).  Functions named
``cum_*`` marshal arguments and call the C entry point of the same name; every
step of the computation runs in the library's CUDA kernels.  PyTorch supplies
device memory and streams only.

Importing this package fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libcumgb.so")

CUM_OK, CUM_EINVAL, CUM_EUNSUPPORTED, CUM_ECUDA, CUM_ETIMEOUT, CUM_EWORKSPACE = range(6)
CUM_F32, CUM_F64 = 0, 1
CUM_PREC_FP64, CUM_PREC_BF16X3, CUM_PREC_FP16X3, CUM_PREC_TF32X3 = 0, 1, 2, 3
CUM_MAX_ORDER = 6
CUM_NOALLOC_WORKSPACE_BYTES = 64 << 20
PRECISIONS = {"fp64": CUM_PREC_FP64, "bf16x3": CUM_PREC_BF16X3, "fp16x3": CUM_PREC_FP16X3, "tf32x3": CUM_PREC_TF32X3}
WS_ALIGN = 256


class CumError(RuntimeError):
    """A non-zero cum_status from the library."""

    def __init__(self, status, what=""):
        self.status = status
        msg = f"{what}: {cum_strerror(status)} (status {status}"
        if status == CUM_ECUDA:
            msg += f", cudaError {cum_last_cuda_error()}"
        super().__init__(msg + ")")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python -m paper_1701_05420_gb300.build` "
            "(or __graft_entry__.build()) before using the library")
    lib = ctypes.CDLL(LIB_PATH)
    c_i, c_i64, c_sz, c_vp, c_dp = ctypes.c_int, ctypes.c_int64, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p
    sig = {
        "cum_num_blocks": (c_i64, [c_i, c_i]),
        "cum_block_rank": (c_i, [c_vp, c_i, c_vp]),
        "cum_block_unrank": (c_i, [c_i64, c_i, c_i, c_vp]),
        "cum_workspace_size": (c_sz, [c_i64, c_i, c_i, c_i, c_i]),
        "cum_center": (c_i, [c_vp, c_i, c_i64, c_i, c_i64, c_i, c_i, c_dp, c_vp, c_sz, c_vp]),
        "cum_moment_blocks": (c_i, [c_i, c_i64, c_i, c_i, c_i, c_dp, c_vp, c_sz, c_vp]),
        "cum_correct": (c_i, [c_i, c_i, c_i, c_dp, c_vp, c_dp, c_vp]),
        "cum_correct_m4": (c_i, [c_i, c_i, c_dp, c_vp, c_dp, c_dp, c_vp]),
        "cum_cumulants": (c_i, [c_vp, c_i, c_i64, c_i, c_i64, c_i, c_i, c_i, c_vp, c_dp, c_vp, c_sz, c_vp]),
        "cum_device_status": (c_i, [c_vp, c_sz, c_vp]),
        "cum_probe_bounded_wait": (c_i, [c_vp, c_sz, c_vp]),
        "cum_plan_info": (c_i, [c_i, c_i64, c_i, c_i, c_i, c_vp]),
        "cum_cumulants_noalloc": (c_i, [c_vp, c_i, c_i64, c_i, c_i64, c_i, c_i, c_i, c_vp, c_dp, c_vp]),
        "cum_batch_plan": (c_i, [c_i, c_vp, c_vp, c_vp, c_i, c_i, c_i, c_vp, c_vp]),
        "cum_batch_bind": (c_i, [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_sz, c_vp]),
        "cum_batch_run": (c_i, [c_vp, c_vp]),
        "cum_batch_info": (c_i, [c_vp, c_vp]),
        "cum_batch_free": (None, [c_vp]),
        "cum_column_sums": (c_i, [c_vp, c_i, c_i64, c_i, c_i64, c_i, c_i, c_dp, c_dp, c_vp, c_sz, c_vp]),
        "cum_mean_from_sums": (c_i, [c_i, c_i64, c_dp, c_dp, c_dp, c_vp]),
        "cum_center_with_mean": (c_i, [c_vp, c_i, c_i64, c_i, c_i64, c_i, c_i, c_dp, c_vp, c_sz, c_vp]),
        "cum_moment_sums": (c_i, [c_i, c_i64, c_i, c_i, c_i, c_dp, c_vp, c_sz, c_vp]),
        "cum_moment_contraction": (c_i, [c_i, c_i64, c_i, c_i, c_i, c_dp, c_vp, c_sz, c_vp]),
        "cum_residual_sums": (c_i, [c_i, c_i, c_i, c_dp, c_vp, c_sz, c_vp]),
        "cum_set_residual_sums": (c_i, [c_i, c_i, c_i, c_dp, c_i64, c_vp, c_sz, c_vp]),
        "cum_finalize": (c_i, [c_i, c_i, c_i, ctypes.c_double, c_dp, c_vp, c_dp, c_vp]),
        "cum_strerror": (ctypes.c_char_p, [c_i]),
        "cum_last_cuda_error": (c_i, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


# ------------------------------------------------------------------ helpers

def _ptr(x):
    """Device (or host) address of a tensor, or None."""
    if x is None:
        return None
    return ctypes.c_void_p(x.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _check(rc, what):
    if rc != CUM_OK:
        raise CumError(rc, what)


def _x_args(X):
    import torch
    if X.dim() != 2 or X.stride(1) != 1:
        raise ValueError("X must be a 2-D tensor with unit column stride (t x n, row-major)")
    if X.dtype == torch.float64:
        dt = CUM_F64
    elif X.dtype == torch.float32:
        dt = CUM_F32
    else:
        raise TypeError("X must be float32 or float64")
    return dt, X.shape[0], X.shape[1], X.stride(0)


def nbar_of(n, b):
    return (n + b - 1) // b


def num_entries(n, d, b):
    """Stored entries of an order-d tensor: cum_num_blocks(nbar, d) * b^d."""
    return cum_num_blocks(nbar_of(n, b), d) * b ** d


# ------------------------------------------------------------------ C ABI, same names

def cum_num_blocks(nbar, d):
    v = lib.cum_num_blocks(int(nbar), int(d))
    if v < 0:
        raise CumError(CUM_EINVAL, "cum_num_blocks")
    return int(v)


def cum_block_rank(j):
    arr = (ctypes.c_int32 * len(j))(*[int(v) for v in j])
    out = ctypes.c_int64(0)
    _check(lib.cum_block_rank(arr, len(j), ctypes.byref(out)), "cum_block_rank")
    return int(out.value)


def cum_block_unrank(rank, d, nbar):
    arr = (ctypes.c_int32 * d)()
    _check(lib.cum_block_unrank(int(rank), int(d), int(nbar), arr), "cum_block_unrank")
    return [int(v) for v in arr]


def cum_workspace_size(t, n, d_max, b, prec):
    return int(lib.cum_workspace_size(int(t), int(n), int(d_max), int(b), int(prec)))


def cum_center(X, b, prec, mean_out, ws, stream=None):
    dt, t, n, ldx = _x_args(X)
    _check(lib.cum_center(_ptr(X), dt, t, n, ldx, int(b), int(prec), _ptr(mean_out), _ptr(ws), ws.numel(),
                          _stream(stream)), "cum_center")


def cum_moment_blocks(d, t, n, b, prec, M_out, ws, stream=None):
    _check(lib.cum_moment_blocks(int(d), int(t), int(n), int(b), int(prec), _ptr(M_out), _ptr(ws), ws.numel(),
                                 _stream(stream)), "cum_moment_blocks")


def cum_correct(d, n, b, M_d, C_lower, C_out, stream=None):
    arr = None
    if C_lower:
        arr = (ctypes.c_void_p * len(C_lower))(*[c.data_ptr() for c in C_lower])
    _check(lib.cum_correct(int(d), int(n), int(b), _ptr(M_d), arr, _ptr(C_out), _stream(stream)), "cum_correct")


def cum_correct_m4(n, b, M_6, C_lower, M_4, C_out, stream=None):
    arr = (ctypes.c_void_p * len(C_lower))(*[c.data_ptr() for c in C_lower])
    _check(lib.cum_correct_m4(int(n), int(b), _ptr(M_6), arr, _ptr(M_4), _ptr(C_out), _stream(stream)),
           "cum_correct_m4")


def cum_cumulants(X, d_max, b, prec, C_out, mean_out, ws, stream=None):
    dt, t, n, ldx = _x_args(X)
    arr = (ctypes.c_void_p * len(C_out))(*[c.data_ptr() for c in C_out])
    _check(lib.cum_cumulants(_ptr(X), dt, t, n, ldx, int(d_max), int(b), int(prec), arr, _ptr(mean_out),
                             _ptr(ws), ws.numel(), _stream(stream)), "cum_cumulants")


def cum_cumulants_noalloc(X, d_max, b, prec, C_out, mean_out, stream=None):
    """cum_cumulants with the library's fixed device workspace (no allocation by
    the caller or the library); see include/cumgb.h for its size limit."""
    dt, t, n, ldx = _x_args(X)
    arr = (ctypes.c_void_p * len(C_out))(*[c.data_ptr() for c in C_out])
    _check(lib.cum_cumulants_noalloc(_ptr(X), dt, t, n, ldx, int(d_max), int(b), int(prec), arr, _ptr(mean_out),
                                     _stream(stream)), "cum_cumulants_noalloc")


class Batch:
    """A planned batch of independent datasets (cum_batch_plan / bind / run / free).

    Bound buffers (inputs, outputs, workspace) are kept referenced here, so they
    stay alive while the plan may run."""

    def __init__(self, ts, ns, bs, d_max, prec, dtype="f32"):
        count = len(ts)
        self.count, self.d_max, self.prec = count, int(d_max), int(prec)
        self.ts = [int(v) for v in ts]
        self.ns = [int(v) for v in ns]
        self.bs = [int(v) for v in bs]
        self.dtype = CUM_F32 if dtype == "f32" else CUM_F64
        tarr = (ctypes.c_int64 * count)(*self.ts)
        narr = (ctypes.c_int * count)(*self.ns)
        barr = (ctypes.c_int * count)(*self.bs)
        handle = ctypes.c_void_p()
        size = ctypes.c_size_t()
        _check(lib.cum_batch_plan(count, tarr, narr, barr, self.d_max, self.prec, self.dtype, ctypes.byref(handle),
                                  ctypes.byref(size)), "cum_batch_plan")
        self.handle = handle
        self.ws_bytes = int(size.value)
        self._keep = None

    def bind(self, X, C, mean=None, ws=None, stream=None):
        """X: list of device tensors (t_i x n_i); C: list of lists C[i][d-2];
        mean: list of device tensors or None; ws: uint8 device tensor."""
        import torch
        if ws is None:
            ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=X[0].device)
        xs = (ctypes.c_void_p * self.count)(*[x.data_ptr() for x in X])
        lds = (ctypes.c_int64 * self.count)(*[x.stride(0) for x in X])
        flat = [c for row in C for c in row]
        cs = (ctypes.c_void_p * len(flat))(*[c.data_ptr() for c in flat])
        ms = None
        if mean is not None:
            ms = (ctypes.c_void_p * self.count)(*[m.data_ptr() for m in mean])
        _check(lib.cum_batch_bind(self.handle, xs, lds, cs, ms, _ptr(ws), ws.numel(), _stream(stream)),
               "cum_batch_bind")
        self._keep = (X, C, mean, ws)
        return ws

    def run(self, stream=None):
        _check(lib.cum_batch_run(self.handle, _stream(stream)), "cum_batch_run")

    def info(self):
        arr = (ctypes.c_int64 * 4)()
        _check(lib.cum_batch_info(self.handle, arr), "cum_batch_info")
        return dict(zip(("datasets", "units", "launches", "ws_bytes"), [int(v) for v in arr]))

    def close(self):
        if self.handle:
            lib.cum_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cum_device_status(ws, stream=None):
    return int(lib.cum_device_status(_ptr(ws), ws.numel(), _stream(stream)))


def cum_column_sums(X, b, prec, shift, sums_out, ws, stream=None):
    dt, t, n, ldx = _x_args(X)
    _check(lib.cum_column_sums(_ptr(X), dt, t, n, ldx, int(b), int(prec), _ptr(shift), _ptr(sums_out), _ptr(ws),
                               ws.numel(), _stream(stream)), "cum_column_sums")


def cum_mean_from_sums(n, t_total, shift, sums, mean_out, stream=None):
    _check(lib.cum_mean_from_sums(int(n), int(t_total), _ptr(shift), _ptr(sums), _ptr(mean_out), _stream(stream)),
           "cum_mean_from_sums")


def cum_center_with_mean(X, b, prec, mean, ws, stream=None):
    dt, t, n, ldx = _x_args(X)
    _check(lib.cum_center_with_mean(_ptr(X), dt, t, n, ldx, int(b), int(prec), _ptr(mean), _ptr(ws), ws.numel(),
                                    _stream(stream)), "cum_center_with_mean")


def cum_moment_sums(d, t, n, b, prec, S_out, ws, stream=None):
    _check(lib.cum_moment_sums(int(d), int(t), int(n), int(b), int(prec), _ptr(S_out), _ptr(ws), ws.numel(),
                               _stream(stream)), "cum_moment_sums")


def cum_moment_contraction(d, t, n, b, prec, M_out, ws, stream=None):
    _check(lib.cum_moment_contraction(int(d), int(t), int(n), int(b), int(prec), _ptr(M_out), _ptr(ws), ws.numel(),
                                      _stream(stream)), "cum_moment_contraction")


def cum_residual_sums(n, b, prec, sums_out, ws, stream=None):
    _check(lib.cum_residual_sums(int(n), int(b), int(prec), _ptr(sums_out), _ptr(ws), ws.numel(), _stream(stream)),
           "cum_residual_sums")


def cum_set_residual_sums(n, b, prec, sums, t_total, ws, stream=None):
    _check(lib.cum_set_residual_sums(int(n), int(b), int(prec), _ptr(sums), int(t_total), _ptr(ws), ws.numel(),
                                     _stream(stream)), "cum_set_residual_sums")


def cum_finalize(d, n, b, scale, S_d, C_lower, C_out, stream=None):
    arr = None
    if C_lower:
        arr = (ctypes.c_void_p * len(C_lower))(*[c.data_ptr() for c in C_lower])
    _check(lib.cum_finalize(int(d), int(n), int(b), float(scale), _ptr(S_d), arr, _ptr(C_out), _stream(stream)),
           "cum_finalize")


def cum_plan_info(d, t, n, b, prec):
    arr = (ctypes.c_int64 * 8)()
    _check(lib.cum_plan_info(int(d), int(t), int(n), int(b), int(prec), arr), "cum_plan_info")
    keys = ("active_tiles", "splits", "units", "tile_m", "tile_n", "chunk", "moment_launches", "center_launches")
    return dict(zip(keys, [int(v) for v in arr]))


def cum_probe_bounded_wait(ws, stream=None):
    _check(lib.cum_probe_bounded_wait(_ptr(ws), ws.numel() * ws.element_size(), _stream(stream)),
           "cum_probe_bounded_wait")


def cum_strerror(status):
    return lib.cum_strerror(int(status)).decode()


def cum_last_cuda_error():
    return int(lib.cum_last_cuda_error())


# ------------------------------------------------------------------ conveniences (torch allocation)

def workspace(t, n, d_max, b, prec, device="cuda"):
    """A uint8 device tensor of cum_workspace_size bytes (torch allocations are 256-byte aligned)."""
    import torch
    size = cum_workspace_size(t, n, d_max, b, prec)
    if size == 0:
        raise CumError(CUM_EUNSUPPORTED, "cum_workspace_size")
    ws = torch.empty(size, dtype=torch.uint8, device=device)
    if ws.data_ptr() % WS_ALIGN:
        raise RuntimeError("workspace allocation is not 256-byte aligned")
    return ws


def cumulants(X, d_max, b, prec=CUM_PREC_FP64, ws=None, stream=None):
    """Cumulant tensors of orders 2..d_max of the rows of X (device tensor t x n).

    Returns ({d: block tensor (float64)}, mean (float64)).  Block layout as in
    include/cumgb.h."""
    import torch
    dt, t, n, _ = _x_args(X)
    if ws is None:
        ws = workspace(t, n, d_max, b, prec, X.device)
    C = [torch.empty(num_entries(n, d, b), dtype=torch.float64, device=X.device) for d in range(2, d_max + 1)]
    mean = torch.empty(n, dtype=torch.float64, device=X.device)
    cum_cumulants(X, d_max, b, prec, C, mean, ws, stream)
    return {d: C[d - 2] for d in range(2, d_max + 1)}, mean


def moments(X, orders, b, prec=CUM_PREC_FP64, ws=None, stream=None):
    """Central moment tensors {d: block tensor} of the rows of X for the given orders."""
    import torch
    dt, t, n, _ = _x_args(X)
    dmax = max(orders)
    if ws is None:
        ws = workspace(t, n, dmax, b, prec, X.device)
    cum_center(X, b, prec, None, ws, stream)
    out = {}
    for d in orders:
        M = torch.empty(num_entries(n, d, b), dtype=torch.float64, device=X.device)
        cum_moment_blocks(d, t, n, b, prec, M, ws, stream)
        out[d] = M
    return out
