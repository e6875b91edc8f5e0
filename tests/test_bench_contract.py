"""The benchmark's host-side pieces, on CPU: the algorithmic KV bytes behind
the decode roofline against a brute-force count of the attention mask, the
traffic record's source check, and the reference arm's JSON line (the FP64
oracle on the host cores), including a non-zero rank that must stay silent."""
import importlib.util
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2606_22984_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _visible_keys(m):
    """Keys each query t sees, counted one by one from the mask definition:
    k <= t, and under the band + sink mask t - k <= W or k < S."""
    n = 0
    for t in range(m.N):
        for k in range(t + 1):
            if m.mask_kind == 0 or t - k <= m.W or k < m.S:
                n += 1
    return n


SHAPES = [
    inputs.ModelShape(20, 2, 32, 4),                               # dense
    inputs.ModelShape(36, 2, 64, 4, mask_kind=1, W=6, S=7),        # band + sink
    inputs.ModelShape(17, 2, 64, 8, mask_kind=1, W=0, S=0),        # the diagonal only
    inputs.ModelShape(20, 2, 64, 4, mask_kind=1, W=3, S=30),       # sink beyond N
    inputs.ModelShape(256, 4, 64, 4, mask_kind=1, W=16, S=17),     # 2D EA L=16
]


@pytest.mark.parametrize("m", SHAPES)
@pytest.mark.parametrize("elem", [2, 4])
def test_decode_bytes_match_the_mask(m, elem):
    b = _bench()
    per_key = 2 * m.d * elem * m.n_layers  # a key and a value per layer
    expect = (_visible_keys(m) + m.N) * per_key  # reads, plus each key/value written once
    assert b.decode_bytes_per_sample(m, elem) == expect


def test_ea2d16_decode_bytes_closed_form():
    """At W = 16, S = 17, queries t <= 33 see all t + 1 keys and later ones
    17 sink + 17 band keys: 595 + 222 * 34 = 8143 key reads, 8.60 MB per
    configuration with the 256 writes in BF16, 140.9 GB at B = 16384."""
    m = inputs.workloads()["ea2d16"].model
    assert _visible_keys(m) == 8143
    per = _bench().decode_bytes_per_sample(m, 2)
    assert per == (8143 + 256) * 2 * 64 * 2 * 4
    assert abs(per * 16384 / 1e9 - 140.91) < 0.01


def test_traffic_record_follows_the_decode_sources():
    b = _bench()
    with open(b.TRAFFIC_FILE) as fh:
        rec = json.load(fh)
    assert rec["traffic_bytes_per_launch"] == rec["dram_bytes_read"] + rec["dram_bytes_write"]
    got = b.captured_traffic(True)
    if rec["source_sha256"] == b.decode_source_hash():
        assert got == float(rec["traffic_bytes_per_launch"])
    else:
        assert got is None  # sources changed since the capture: no traffic claimed
    assert b.captured_traffic(False) is None


def _run_reference(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--steps", "1", "--warmup", "3", "--cpu-seconds", "0.5"],
                          capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)


def test_reference_arm_json_line():
    r = _run_reference({"RANK": "0"})
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["unit"] == "configs/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 3
    assert line["config"]["workload"] == inputs.workloads()["ea2d16"].name
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_stay_silent():
    r = _run_reference({"RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
