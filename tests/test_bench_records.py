"""Host logic of the benchmark on CPU: the recorded ncu figures that the
JSON line quotes (each names a source file and kernel that exist, and is
dropped once that file's hash no longer matches), the per-V-cycle
bandwidth arithmetic, and the reference arm's line (the oracle timed on
the host cores) on a small workload."""
import hashlib
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _records(name):
    with open(os.path.join(ROOT, "profiles", name)) as f:
        return json.load(f)


@pytest.mark.parametrize("name", ["traffic.json", "fp64_ops.json"])
def test_records_name_existing_sources_kernels_and_summaries(name):
    for key, rec in _records(name).items():
        src = os.path.join(ROOT, rec["source"])
        assert os.path.isfile(src), (key, rec["source"])
        with open(src) as f:
            assert rec["function"] in f.read(), (key, rec["function"])
        assert os.path.isfile(os.path.join(ROOT, rec["summary"])), (key, rec["summary"])
        assert len(rec["source_sha256"]) == 64


def _write(tmp_path, name, recs):
    p = tmp_path / name
    p.write_text(json.dumps(recs))
    return str(p)


def test_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    src = "paper_1807_10504_gb300/csrc/mg.cu"
    with open(os.path.join(ROOT, src), "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()
    recs = {"ok": {"function": "k_smooth2t_f32", "source": src, "source_sha256": sha,
                   "dram_bytes_per_cell": 31.5},
            "stale": {"function": "k_smooth2t_f32", "source": src, "source_sha256": "0" * 64,
                      "dram_bytes_per_cell": 31.5}}
    monkeypatch.setattr(bench, "TRAFFIC", _write(tmp_path, "traffic.json", recs))
    assert bench.traffic_per_launch("ok", 1 << 20) == 31.5 * (1 << 20)
    assert bench.traffic_per_launch("stale", 1 << 20) is None
    assert bench.traffic_per_launch("absent", 1 << 20) is None


def test_fp64_record_follows_the_source_hash(tmp_path, monkeypatch):
    src = "paper_1807_10504_gb300/csrc/grid.cu"
    with open(os.path.join(ROOT, src), "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()
    recs = {"k_predictor": {"function": "k_predictor", "source": src, "source_sha256": sha,
                            "fp64_flops_per_unit": 35.0},
            "k_old": {"function": "k_predictor", "source": src, "source_sha256": "f" * 64}}
    monkeypatch.setattr(bench, "FP64_OPS", _write(tmp_path, "fp64_ops.json", recs))
    assert bench.fp64_record("k_predictor")["fp64_flops_per_unit"] == 35.0
    assert bench.fp64_record("k_old") is None


def test_per_vcycle_bandwidth_and_fp64_rate():
    cells = 1 << 20
    out = bench.per_vcycle({"ms": 1.0, "cycles": 10}, cells, {"hbm_gbs": 5000.0}, 1.25, True)
    assert out["us"] == pytest.approx(100.0)
    # 112 B per fine cell over 100 us
    assert out["fused_112B"]["GB_s"] == pytest.approx(112.0 * cells / 100e-6 / 1e9)
    assert out["fused_112B"]["frac_hbm"] == pytest.approx(out["fused_112B"]["GB_s"] / 5000.0)
    assert out["unfused_283B"]["GB_s"] == pytest.approx(283.0 * cells / 100e-6 / 1e9)
    tf = bench.VCYCLE_FP64_FLOPS * cells / 100e-6 / 1e12
    assert out["fp64"]["tflops"] == pytest.approx(tf)
    assert out["fp64"]["frac"] == pytest.approx(tf / 1.25)
    # (4 sweeps x 8 + 5 + 7) x 4/3 + 15 FP64 operations per fine cell
    assert bench.VCYCLE_FP64_FLOPS == pytest.approx(44.0 * 4.0 / 3.0 + 15.0)
    assert "fp64" not in bench.per_vcycle({"ms": 1.0, "cycles": 10}, cells,
                                          {"hbm_gbs": 5000.0}, 1.25, False)


def test_host_info_reads_cores_and_model():
    info = bench.host_info()
    assert info["nproc"] >= 1 and isinstance(info["cpu_model"], str)


def test_reference_arm_line_on_a_small_workload():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "static64",
                        "--steps", "2", "--warmup", "1"], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "steps/s"
    assert line["steps"] == 2 and line["warmup"] == 1 and line["value"] > 0
    assert line["higher_is_better"] is True and line["config"]["workload"] == "static64"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert cb["nproc"] >= 1 and "sample" in cb
    assert line["e2e"] == {"value": line["value"], "unit": "steps/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
