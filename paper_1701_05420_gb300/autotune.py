"""Choice of the block side b per dataset, from measurements cached on disk.

The paper tunes b by hand and finds b = 2 fastest on its CPUs (Sec. 5.2.1).
Here b also changes the tile staircase of the GPU contraction, so the best b
depends on n, t, the orders and the precision.  The tuner:

* ranks candidate b values (divisor-friendly sides up to n) with a cost model
  built from the library's own execution plan (``cum_plan_info``: work units x
  samples per unit, plus the stored entries the correction touches);
* measures the best few candidates on the GPU for each class of datasets (same
  n, t rounded to a power of two, same orders and precision), timing
  ``cum_cumulants`` with CUDA events on synthetic data of that shape;
* caches the winner per class in a JSON file keyed by the GPU's name.

``measure`` can be replaced (the tests drive the tuner with a fake timer).
"""
from __future__ import annotations

import json
import math
import os

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "cumgb", "autotune.json")
CANDIDATES = (2, 3, 4, 6, 8, 12, 16)


def t_bucket(t):
    """Class of a sample count: the nearest power of two (log2, rounded)."""
    return int(round(math.log2(max(int(t), 1))))


def candidates(n, prec):
    """Block sides worth trying for n variables (the tensor-core paths stage at
    most 256 variables, padded to a multiple of b)."""
    out = [b for b in CANDIDATES if b <= max(n, 2)]
    if prec != 0:
        out = [b for b in out if -(-n // b) * b <= 256]
    return out or [1]


def model_cost(t, n, b, d_max, prec, plan_info=None):
    """Relative cost of computing orders 2..d_max with block side b: contraction
    work units x their samples (tensor-core tiles are 128 x 128, FP64 tiles
    64 x 64), plus the correction's stored entries of orders >= 4 x the number of
    partition terms."""
    import paper_1701_05420_gb300 as cum
    info = plan_info or cum.cum_plan_info
    terms = {4: 3, 5: 10, 6: 40}
    cost = 0.0
    for d in range(2, d_max + 1):
        p = info(d, t, n, b, prec)
        cost += p["units"] * p["chunk"] * p["tile_m"] * p["tile_n"]
        if d >= 4:
            cost += 8.0 * cum.num_entries(n, d, b) * terms[d]
    return cost


class AutoTuner:
    def __init__(self, d_max, prec, cache_path=DEFAULT_CACHE, measure=None, device_name=None, shortlist=3):
        self.d_max, self.prec = int(d_max), int(prec)
        self.cache_path = cache_path
        self.measure = measure or self._measure_gpu
        self.device_name = device_name
        self.shortlist = shortlist
        self.cache = {}
        if cache_path and os.path.exists(cache_path):
            try:
                with open(cache_path) as f:
                    self.cache = json.load(f)
            except (OSError, ValueError):
                self.cache = {}

    def _device(self):
        if self.device_name is None:
            import torch
            self.device_name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
        return self.device_name

    def key(self, n, t):
        return f"{self._device()}|prec{self.prec}|d{self.d_max}|n{int(n)}|t2^{t_bucket(t)}"

    def _measure_gpu(self, t, n, b):
        """Median CUDA-event time (ms) of cum_cumulants on synthetic data of this shape."""
        import torch

        import paper_1701_05420_gb300 as cum
        import numpy as np
        rng = np.random.default_rng(12345)
        X = torch.from_numpy(rng.standard_t(5.0, size=(int(t), int(n))).astype(np.float32)).cuda()
        ws = cum.workspace(t, n, self.d_max, b, self.prec)
        C = [torch.empty(cum.num_entries(n, d, b), dtype=torch.float64, device="cuda")
             for d in range(2, self.d_max + 1)]
        cum.cum_cumulants(X, self.d_max, b, self.prec, C, None, ws)
        times = []
        for _ in range(3):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            cum.cum_cumulants(X, self.d_max, b, self.prec, C, None, ws)
            e.record()
            torch.cuda.synchronize()
            times.append(s.elapsed_time(e))
        return sorted(times)[1]

    def choose(self, t, n):
        k = self.key(n, t)
        if k in self.cache:
            return int(self.cache[k]["b"])
        tt = 2 ** t_bucket(t)
        cands = candidates(n, self.prec)
        ranked = sorted(cands, key=lambda b: model_cost(tt, n, b, self.d_max, self.prec))[: self.shortlist]
        timed = {b: float(self.measure(tt, n, b)) for b in ranked}
        best = min(timed, key=timed.get)
        self.cache[k] = {"b": int(best), "ms": timed}
        self._save()
        return int(best)

    def choose_all(self, shapes):
        """b for every (t, n) in shapes."""
        return [self.choose(t, n) for (t, n) in shapes]

    def _save(self):
        if not self.cache_path:
            return
        os.makedirs(os.path.dirname(self.cache_path), exist_ok=True)
        tmp = self.cache_path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(self.cache, f, indent=1, sort_keys=True)
        os.replace(tmp, self.cache_path)
