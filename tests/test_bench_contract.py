"""The benchmark's output contract, checked on the CPU: the reference arm
(the FP64 oracle timed on the host cores) prints one JSON line with the
fields every line of bench.py carries, and the workload it names is the one
the seeded input recipe builds."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _reference_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600, check=True).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out
    return json.loads(lines[0])


def test_reference_arm_line():
    d = _reference_line()
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1
    assert d["unit"] == "triplets/s" and d["higher_is_better"] is True and d["value"] > 0
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_headline_workload_matches_recipe():
    """The headline is the largest single-GPU configuration: ATM energy and
    forces at n = 16384, uniform in a cube of side 20, seed 6."""
    import bench
    import synth
    w = synth.WORKLOADS[bench.WORKLOAD]
    cfg = bench.config_block()
    assert cfg["n"] == w["n"] == 16384 and w["side"] == 20.0 and w["seed"] == 6
    assert cfg["triples"] == bench.triples(w["n"]) == 16384 * 16383 * 16382 // 6
    x = synth.make_points(bench.WORKLOAD)
    assert x.shape == (16384, 3) and x.dtype.name == "float32"
    assert float(x.min()) >= 0.0 and float(x.max()) < 20.0
    rows = bench.headline_cpu_rows(16384, 4)
    assert len(rows) == 4 and all(5e6 < bench.row_triples(16384, i) < 2e7 for i in rows)


@pytest.mark.parametrize("name", ["cover2_n16384", "cover3_n1024", "cover4_n256", "edm_n65536_d64",
                                  "atm_n1024", "atm_n4096", "stress_n65536_d64", "cover2_n12000",
                                  "edm_n49152_d64", "atm_n3000", "atm_n12000"])
def test_rows_are_registered(name):
    import bench
    assert name in bench.ROWS


def test_stated_traffic(tmp_path, monkeypatch):
    """roofline.traffic comes from a committed ncu summary only while the
    kernel's source file is the one captured."""
    import hashlib
    import bench
    src = tmp_path / "k.cu"
    src.write_text("kernel v1\n")
    digest = hashlib.sha256(src.read_bytes()).hexdigest()
    prof = tmp_path / "prof"
    prof.mkdir()
    (prof / "k.md").write_text(f"# k\n<!-- bench: source=k.cu sha256={digest} traffic_bytes_per_launch=1.5e9 "
                               f"scale=captured_at_n=4096 -->\n")
    monkeypatch.setattr(bench, "PROFILES", str(prof))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    value, note = bench.stated_traffic("k.md")
    assert value == 1.5e9 and "captured at n=4096" in note
    src.write_text("kernel v2\n")
    assert bench.stated_traffic("k.md")[0] is None
    assert bench.stated_traffic("missing.md")[0] is None


def test_edm_error_report(monkeypatch):
    """The benchmark's EDM error report on a known output: the FP32 rounding
    of the exact squared distances reports at most 2^-24 relative error and
    an exactly-zero diagonal; a perturbed entry shows up as the maximum."""
    import numpy as np
    import torch
    import bench
    import synth
    monkeypatch.setattr(torch.Tensor, "cuda", lambda self, *a, **k: self)
    xh = synth.normal(300, 16, 7)
    x64 = xh.astype(np.float64)
    i, j = np.tril_indices(len(xh))          # row-major lower: index i(i+1)/2 + j
    exact = ((x64[i] - x64[j]) ** 2).sum(axis=1)
    o = torch.from_numpy(exact.astype(np.float32))
    r = bench._edm_error(torch, o, xh, seed=5, count=20000, tile=32)
    assert r["diagonal_exact_zero"]
    for part in ("sampled", "diagonal_tiles"):
        assert r[part]["pairs"] == 20000
        assert r[part]["max_rel"] <= 2.0 ** -24 and r[part]["p99_rel"] <= r[part]["max_rel"]
    bad = o.clone()
    pr = synth.sample_pairs(20000, len(xh), 5)
    k = int(pr[0, 0] * (pr[0, 0] + 1) // 2 + pr[0, 1])
    if pr[0, 0] != pr[0, 1]:
        bad[k] *= 1.001
        assert bench._edm_error(torch, bad, xh, seed=5, count=20000, tile=32)["sampled"]["max_rel"] > 9e-4
