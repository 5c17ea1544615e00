"""The block-side tuner's host logic (no GPU): candidate sets, the plan-based
cost model, measurement of a shortlist, and the on-disk cache."""
import json

from paper_1701_05420_gb300 import autotune


def test_candidates_respect_limits():
    assert autotune.candidates(1, 3) == [2]
    assert 16 in autotune.candidates(96, 3)
    assert all(-(-255 // b) * b <= 256 for b in autotune.candidates(255, 3))
    assert autotune.candidates(5, 0) == [2, 3, 4]


def test_model_cost_follows_stored_entries():
    # the contraction's work follows the stored entries, which shrink with b (less
    # diagonal-block redundancy): the model prefers b = 2 at n = 96, as the paper's
    # CPU timing did (Sec. 5.2.1), and grows steadily with b
    c = {b: autotune.model_cost(2 ** 16, 96, b, 4, 3) for b in (2, 4, 8, 16)}
    assert min(c, key=c.get) == 2
    assert c[2] < c[4] < c[8] < c[16]


def test_choose_measures_shortlist_and_caches(tmp_path):
    calls = []

    def fake_measure(t, n, b):
        calls.append((t, n, b))
        return {2: 5.0, 3: 4.0, 4: 1.0, 6: 2.0, 8: 3.0}.get(b, 9.0)

    path = tmp_path / "cache.json"
    tuner = autotune.AutoTuner(4, 3, cache_path=str(path), measure=fake_measure, device_name="fake", shortlist=7)
    b = tuner.choose(50000, 48)
    assert b == 4
    assert {c[2] for c in calls} == set(autotune.candidates(48, 3))
    assert all(t == 2 ** autotune.t_bucket(50000) for t, _, _ in calls)
    # same class: served from the cache, no new measurement
    n_calls = len(calls)
    assert tuner.choose(60000, 48) == 4 and len(calls) == n_calls
    # a new tuner reads the cache from disk
    data = json.loads(path.read_text())
    assert any(k.startswith("fake|prec3|d4|n48") for k in data)
    tuner2 = autotune.AutoTuner(4, 3, cache_path=str(path), measure=lambda *a: 1 / 0, device_name="fake")
    assert tuner2.choose(50000, 48) == 4


def test_choose_all_shapes(tmp_path):
    tuner = autotune.AutoTuner(4, 1, cache_path=str(tmp_path / "c.json"), measure=lambda t, n, b: float(b),
                               device_name="fake", shortlist=2)
    bs = tuner.choose_all([(5000, 16), (200000, 96), (5000, 16)])
    assert len(bs) == 3 and bs[0] == bs[2]
