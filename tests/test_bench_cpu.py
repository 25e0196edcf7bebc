"""The benchmark's reference arm (the oracle timed on the host cores) prints
the one JSON line of the benchmark contract, here on a small grid."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                          "--warmup", "1", "--size", "16"], cwd=ROOT, capture_output=True,
                         text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "cells/s" and d["value"] > 0
    for key in ("metric", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "dtype", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert "16^3" in d["config"]["workload"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_reference_and_gpu_arms_name_the_same_config():
    # the two arms print identical config dicts for one size, so that their
    # lines compare like for like
    sys.path.insert(0, ROOT)
    import bench
    src = open(os.path.join(ROOT, "bench.py")).read()
    want = ('"config": {"workload": WORKLOAD.format(n=n), "cells": N, "tol": TOL, '
            '"l2": L2_NOTE}')
    assert src.count(want) == 2, "both arms build config the same way"
    assert bench.workload_seed(512) == 3 and bench.workload_seed(256) == 2


def test_stored_traffic_follows_the_kernel_source(tmp_path, monkeypatch):
    # a DRAM figure from an ncu capture is reported only while the kernel's
    # source region (and the shared header) is the one it was taken on; a
    # capture on another size is scaled by the cell count
    import shutil
    sys.path.insert(0, ROOT)
    import bench
    n256 = 256 ** 3
    t256, note = bench.stored_traffic("rbgs_sweep_tma_f32", n256)
    assert t256 is not None and "this size" in note
    t512, note = bench.stored_traffic("rbgs_pass_f64", 8 * n256)
    assert t512 is not None and "this size" in note
    t, note = bench.stored_traffic("rbgs_pass_f64", n256)     # captured at 512^3 only
    assert "scaled" in note and abs(t - t512 / 8) <= 1
    src = tmp_path / "paper_1008_2801_gb300" / "csrc"
    src.mkdir(parents=True)
    for f in ("kernels.cu", "sweep_tma.cu", "common.cuh"):
        shutil.copy(os.path.join(ROOT, "paper_1008_2801_gb300", "csrc", f), src / f)
    shutil.copytree(os.path.join(ROOT, "profiles"), tmp_path / "profiles")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.stored_traffic("rbgs_pass_f64", n256)[0] is not None
    assert bench.stored_traffic("rbgs_sweep_tma_f32", n256)[0] is not None
    text = (src / "kernels.cu").read_text()
    a, b = bench.TRAFFIC_REGIONS["rbgs_pass_f64"]
    i = text.index(a) + len(a)
    (src / "kernels.cu").write_text(text[:i] + "\n// edited\n" + text[i:])
    assert bench.stored_traffic("rbgs_pass_f64", n256)[0] is None           # its region changed
    assert bench.stored_traffic("rbgs_sweep_tma_f32", n256)[0] is not None  # the other did not
    (src / "kernels.cu").write_text(text)
    (src / "sweep_tma.cu").write_text((src / "sweep_tma.cu").read_text() + "\n")
    assert bench.stored_traffic("rbgs_sweep_tma_f32", n256)[0] is None      # its file changed
    assert bench.stored_traffic("rbgs_pass_f64", n256)[0] is not None
    (src / "common.cuh").write_text((src / "common.cuh").read_text() + "\n")
    assert bench.stored_traffic("rbgs_pass_f64", n256)[0] is None       # the shared header changed
