"""The reference arm of bench.py (the FP64 oracle on the host cores): its one
JSON line carries the headline's metric, config, unit and direction, W
untimed and K timed steps, and the keys the line's contract asks for.
CPU only (a small per-step sample)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _run(*args):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        *args], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


def test_reference_line_matches_the_headline():
    line = _run("--steps", "2", "--warmup", "1", "--ref-side", "64")
    metric, config = bench.headline_meta(1)
    assert line["impl"] == "reference"
    assert line["metric"] == metric
    assert line["config"] == config
    assert line["unit"] == "Mpx/s" and line["higher_is_better"] is True
    assert line["steps"] == 2 and line["warmup"] == 1
    assert line["value"] > 0 and line["ms_per_step"] > 0
    # value is the timed steps' pixels over their time
    assert abs(line["value"] - 64 * 64 / (line["ms_per_step"] * 1e-3) / 1e6) < 1e-6 * line["value"] + 1e-9
    cb = line["cpu_baseline"]
    # a 64x64 sample is one group: one worker
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"]
    assert "64x64" in cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_sample_is_sized_to_the_run():
    """Without --ref-side the per-step sample shrinks as K + W grows, so the
    whole run stays within a few minutes of oracle time on the cores it
    uses (each group's crop is about 2.3 times the group)."""
    for cores in (1, 16):
        sides = [bench.reference_side(k, 10, cores=cores) for k in (1, 10, 50, 200, 1000)]
        assert sides == sorted(sides, reverse=True)
        for k, w in ((200, 10), (50, 3), (20, 5), (3, 3)):
            s = bench.reference_side(k, w, cores=cores)
            used = max(1, min(cores, (s // bench.GROUP) ** 2))
            assert s % bench.GROUP == 0
            assert s == 256 or (k + w) * s * s * 2.3 * bench.ORACLE_S_PER_PX / used <= 150.0
        assert bench.reference_side(10 ** 6, 0, cores=cores) == 256     # floor
    assert bench.reference_side(3, 3, cores=16) > bench.reference_side(3, 3, cores=1)
