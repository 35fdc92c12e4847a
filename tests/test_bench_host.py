"""Host side of the benchmark contract on CPU: the reference arm (the oracle timed on the
host cores) prints one JSON line with the keys the driver reads, and its sample shrinks
with the number of steps so that a run stays near two minutes."""
import argparse
import io
import json
from contextlib import redirect_stdout

import bench


def test_reference_sample_size_bounds_the_run():
    assert bench.reference_sample_size(1, 0) == 1024
    for steps, warmup in ((3, 3), (10, 3), (40, 3), (200, 10)):
        s = bench.reference_sample_size(steps, warmup)
        assert s in (1024, 768, 512, 384, 256)
        if s > 256:
            assert (steps + warmup) * 25.0 * (s / 1024.0) ** 2 <= 150.0


def test_reference_arm_json_line(monkeypatch):
    monkeypatch.setattr(bench, "reference_sample_size", lambda steps, warmup: 256)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    args = argparse.Namespace(steps=1, warmup=0, gpus=1)
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    lines = [ln for ln in buf.getvalue().splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["unit"] == "pairs/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "pairs/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    # a 256^2 sample is credited as (256 / 1024)^2 of a pair
    assert abs(d["config"]["pairs_per_step"] - 1 / 16) < 1e-12
