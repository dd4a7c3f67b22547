"""bench.py's command-line contract on the CPU: the reference arm (the FP64 oracle on the host
cores) prints exactly one JSON line with the keys the measurement reports carry, and the
arguments are checked (at least 3 warm-up steps)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
METRIC = "gridding/degridding G grid-point updates/s and % roofline at stated grid error"


def _bench(*args, timeout=600):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                          text=True, timeout=timeout)


def test_reference_arm_prints_one_complete_line():
    r = _bench("--impl", "reference", "--steps", "1", "--warmup", "3")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    x = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in x, k
    assert x["impl"] == "reference" and x["metric"] == METRIC
    assert (x["n_gpus"], x["steps"], x["warmup"]) == (1, 1, 3)
    assert x["value"] > 0 and x["ms_per_step"] > 0 and x["higher_is_better"] is True
    assert x["config"]["workload"].startswith("wproj_2k")
    cb = x["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == x["value"] and cb["sample"]
    e = x["e2e"]
    assert e["value"] == x["value"] and e["unit"] == x["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_fewer_than_three_warmup_steps_are_rejected():
    r = _bench("--impl", "reference", "--steps", "1", "--warmup", "2", timeout=120)
    assert r.returncode != 0 and "warmup" in r.stderr


def test_channel_groups_are_split_over_launches_at_the_entry_limit():
    """bench.py packs the batched workload's channel groups into gridder launches whose entries
    fit 32-bit indices; a group is never split, and a group over the limit is an error."""
    import pytest
    sys.path.insert(0, ROOT)
    import bench
    assert bench.split_launches([]) == []
    assert bench.split_launches([3, 4, 2], limit=10) == [[0, 1, 2]]
    assert bench.split_launches([6, 5, 4], limit=10) == [[0], [1, 2]]
    assert bench.split_launches([10, 1, 9, 1], limit=10) == [[0], [1, 2], [3]]
    assert bench.split_launches([0, 0], limit=0) == [[0, 1]]
    # the batched workload's 8 groups of about 163 M entries fit one launch
    assert bench.split_launches([163_000_000] * 8) == [list(range(8))]
    assert bench.split_launches([700_000_000] * 4) == [[0, 1, 2], [3]]
    with pytest.raises(ValueError, match="group 1"):
        bench.split_launches([5, 11], limit=10)
