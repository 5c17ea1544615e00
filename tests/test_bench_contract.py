"""CPU checks of bench.py's output contract: the reference arm (the oracle on
the host cores) prints one JSON line with the required keys, other ranks print
nothing, and the helper that counts the correction's FP64 work matches the
forms the library runs."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(args, env_extra=None):
    env = dict(os.environ)
    for k in ("RANK", "LOCAL_RANK", "WORLD_SIZE"):
        env.pop(k, None)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _bench(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    j = json.loads(lines[0])
    assert j["impl"] == "reference" and j["value"] > 0 and j["unit"] == "block-entries*samples/s"
    assert j["n_gpus"] == 1 and j["steps"] == 1 and j["warmup"] == 0
    assert j["higher_is_better"] is True and j["scaling"] == "weak" and j["vs_baseline"] is None
    assert j["config"]["workload"] == "high-order"
    cb = j["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == j["value"]
    assert j["e2e"] == {"value": j["value"], "unit": j["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_nothing():
    r = _bench(["--impl", "reference", "--steps", "1", "--warmup", "0"], {"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_correction_flops_follow_the_library_forms():
    sys.path.insert(0, ROOT)
    saved = sys.argv
    sys.argv = ["bench.py"]
    try:
        import bench
    finally:
        sys.argv = saved
    # per entry: 2 per two-part partition + 2; order 6 adds 5 groups of 7 for
    # the three-pair partitions unless the order-4 moment replaces them
    assert bench.correction_flops(4, 1) == 2 * 3 + 2
    assert bench.correction_flops(5, 1) == 2 * 10 + 2
    assert bench.correction_flops(6, 1) == 2 * 25 + 35 + 2
    assert bench.correction_flops(6, 1, moment_form=True) == 2 * 25 + 2


def test_sampled_entry_offsets_match_the_tests_reading_of_block_storage():
    """bench.py gathers the sampled entries of the timed step's output through
    the C ABI's block rank; the offsets equal those of the tests' independent
    colex-sort reading of the storage layout."""
    import numpy as np

    import blocks
    import paper_1701_05420_gb300 as cum
    import synth
    sys.path.insert(0, ROOT)
    saved = sys.argv
    sys.argv = ["bench.py"]
    try:
        import bench
    finally:
        sys.argv = saved
    for n, b, d in ((48, 4, 6), (60, 6, 4), (13, 3, 5), (7, 1, 3)):
        idx = synth.sample_indices(n, d, 200, seed=d + n)
        np.testing.assert_array_equal(bench.entry_offsets(cum, idx, n, b), blocks.entry_offsets(idx, n, b))
    # the leading N_SPECIAL entries are compared against their moments, the rest normwise
    k = bench.N_SPECIAL
    got = np.concatenate([np.full(k, 1.0), [1.0, 2.0, 3.0]])
    ref = np.concatenate([np.full(k, 1.5), [1.0, 2.0, 4.0]])
    rec = bench.error_record(got, ref, np.full(k, 2.0))
    assert abs(rec["relF"] - 1.0 / np.sqrt(21.0)) < 1e-15 and rec["relMax"] == 0.25 and rec["entries"] == 3
    assert abs(rec["special_vs_moments"] - 0.25) < 1e-15 and rec["special_entries"] == k
