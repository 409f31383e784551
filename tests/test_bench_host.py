"""Host logic of bench.py (no GPU): the algorithmic byte counts of the roofline,
the lookup of the profiled DRAM traffic, and the JSON line of the reference arm."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_algorithmic_bytes_per_format():
    E, N = 1000, 100
    staged = bench.algorithmic_bytes({"step_kernel": 3, "step_gathers": 400}, E, N)
    assert staged == pytest.approx(E * 6 + 400 * 8 + N * 36.2)
    plain = bench.algorithmic_bytes({"step_kernel": 1, "step_gathers": E}, E, N)
    assert plain == pytest.approx(E * 12 + N * 36.2)
    # the per-node figures of the spiking models extend the FitzHugh-Nagumo one
    assert bench.HH_NODE_BYTES == pytest.approx(bench.IZH_NODE_BYTES - 0.2 + 32 + 4 / 33, abs=0.01)


def test_traffic_is_taken_only_for_the_profiled_source_and_tiling(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_hash", lambda: "abc")
    p = prof / "k_step_staged_roofline.json"
    p.write_text(json.dumps({"kernel_hash": "abc", "dram_bytes_per_launch_by_grid": {"4002": 5.0e8}}))
    assert bench.traffic_per_launch("k_step_staged", "roofline", 4002) == 5.0e8
    assert bench.traffic_per_launch("k_step_staged", "roofline", 4350) is None
    p.write_text(json.dumps({"kernel_hash": "abc", "dram_bytes_per_launch": 6.0e8}))
    assert bench.traffic_per_launch("k_step_staged", "roofline", 1) == 6.0e8
    p.write_text(json.dumps({"kernel_hash": "old", "dram_bytes_per_launch": 6.0e8}))
    assert bench.traffic_per_launch("k_step_staged", "roofline", 1) is None
    assert bench.traffic_per_launch("k_step", "roofline", 1) is None


def test_kernel_hash_ignores_comments_and_layout_only(tmp_path, monkeypatch):
    import shutil
    src = os.path.join(ROOT, "paper_0908_3934_b300", "csrc")
    dst = tmp_path / "paper_0908_3934_b300" / "csrc"
    shutil.copytree(src, dst)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_hash()
    f = dst / "k_step_staged.cu"
    code = f.read_text()
    f.write_text("// a new comment\n/* and a\n block */\n" + code.replace(";\n", ";   \n", 3))
    assert bench.kernel_hash() == h0
    f.write_text(code.replace("kThreadsL2 = 1280", "kThreadsL2 = 1024"))
    assert bench.kernel_hash() != h0


def test_reference_arm_prints_one_contract_line():
    env = dict(os.environ, PYTHONPATH=ROOT, OMP_NUM_THREADS="1")
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "tiny",
                          "--steps", "4", "--warmup", "3"], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["higher_is_better"] is True and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1


def test_config_names_the_workload_as_generated():
    from types import SimpleNamespace
    from paper_0908_3934_b300 import netgen
    tiny = bench.config_of(SimpleNamespace(workload="tiny"), netgen.tiny(), 1)
    assert "no background" in tiny["workload"] and "ring sized to the delays" in tiny["workload"]
    big = bench.config_of(SimpleNamespace(workload="large"), netgen.large(n=2000, mean_deg=20.0), 2)
    assert "5 Hz background" in big["workload"] and "ring 256" in big["workload"]
    assert big["replicas"] == 2 and big["parallelism"] == "replicas2" and big["dt_ms"] == 0.05


def test_printed_line_drops_details_and_rounds():
    line = {"value": 1.23456789e11, "config": {"workload": "x"}, "steps": 20,
            "test_set": {"rtf_min": 12.3456, "details_networks": [{"name": "a"}]}, "details_layout": {"grid": 1}}
    out = bench.compact(bench.strip_details(line))
    assert out == {"value": 1.235e11, "config": {"workload": "x"}, "steps": 20, "test_set": {"rtf_min": 12.35}}


def test_survey_bytes_are_format_independent():
    assert bench.survey_bytes(1000, 100) == pytest.approx(1000 * 14 + 100 * 36.2)


def test_all_cores_oracle_run_times_independent_copies():
    """The all-cores leg of cpu_baseline: one spawned copy of the plain oracle sample
    per core (bounded by the memory allowance), the copies' edge-updates over the
    slowest copy's time; the same network as the one-thread sample."""
    spec = bench.workload("tiny", 0)
    one = bench.cpu_baseline(spec, 50)
    ac = bench.cpu_baseline_all_cores("tiny", spec, 50, bytes_per_copy=1e8)
    assert 1 <= ac["cores"] <= (os.cpu_count() or 1)
    assert ac["kind"] == "oracle" and ac["unit"] == one["unit"]
    assert ac["value"] > 0 and ac["seconds"] > 0
    assert f"{ac['cores']} independent copies" in ac["sample"]
