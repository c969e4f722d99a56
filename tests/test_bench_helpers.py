"""Host logic of bench.py: the capture-staleness digest, the committed traffic lookup and
the algorithmic byte counts (CPU only)."""
import argparse
import json
import os
import shutil

import pytest

import bench


def argparse_ns(n, m, bins):
    return argparse.Namespace(n=n, m=m, bins=bins)


def test_code_digest_ignores_comments_and_whitespace(tmp_path):
    a, b, c = tmp_path / "a.cu", tmp_path / "b.cu", tmp_path / "c.cu"
    a.write_text("int f(int x) { return x + 1; }  // one\n")
    b.write_text("/* header */\nint f(int x)\n{\n    return x + 1;  // other comment\n}\n")
    c.write_text("int f(int x) { return x + 2; }\n")
    assert bench.code_digest(str(a)) == bench.code_digest(str(b))
    assert bench.code_digest(str(a)) != bench.code_digest(str(c))


def test_traffic_is_per_launch_and_null_once_the_kernel_changed(tmp_path, monkeypatch):
    doc = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    e = doc["stages"]["gtg"]
    # a copy of the tree whose grid source is the committed one, then an edited one
    os.makedirs(tmp_path / "profiles")
    shutil.copy(os.path.join(bench.ROOT, "profiles", "traffic.json"), tmp_path / "profiles")
    src = tmp_path / e["source"]
    os.makedirs(src.parent)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    shutil.copy(os.path.join(os.path.dirname(bench.__file__), e["source"]), src)
    if bench.code_digest(str(src)) != e["code_sha256"]:
        pytest.skip("the grid kernel changed since the committed capture (traffic reported as null)")
    assert bench.measured_traffic("gtg", 32) == pytest.approx(e["bytes_per_step"] / 32)
    with open(src, "a") as f:
        f.write("\nstatic int changed_code = 1;\n")
    assert bench.measured_traffic("gtg", 32) is None
    assert bench.measured_traffic("no_such_stage", 1) is None


def test_apply_bytes_follow_the_stage_sum():
    info = {"K": 10_523_716_232}
    n, P, M, tiles, PW = 4096, 32, 50_000_000, 158_300, 46
    sb = bench.stage_bytes(info, n, P, M, tiles, PW)
    patches = 8.0 * tiles * PW * PW
    assert sb["apply_per_step"] == pytest.approx(8 * info["K"] + 16 * M + 3 * patches + P * 120 * n * n)
    per_bin_fft = sb["fwd_rows"] + sb["fwd_cols"] + sb["inv_rows"]
    assert sb["apply_per_step"] == pytest.approx(sb["gtg_per_step"] + sb["inv_cols_per_step"] + P * per_bin_fft)


def test_workload_label_names_the_sizes_run():
    full, small = argparse_ns(4096, 50_000_000, 32), argparse_ns(256, 20000, 4)
    assert bench.workload_name(full) == bench.WORKLOAD
    assert "256x256 image" in bench.workload_name(small) and "20000 visibilities" in bench.workload_name(small)


def test_reference_arm_prints_one_contract_line():
    # the reference arm times the FP64 oracle on the host cores (no GPU involved)
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference",
                        "--n", "256", "--m", "20000", "--bins", "4", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=600, cwd=bench.ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["ms_per_step"] == pytest.approx(1000.0 / d["value"])
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 1, 0)
    assert d["config"]["workload"] == bench.workload_name(argparse_ns(256, 20000, 4))
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
