"""The bench's reference arm (the FP64 oracle timed on the host cores) prints one JSON line that
keeps the bench contract: the same metric, unit and config as the GPU arm, plus the CPU-baseline
and end-to-end blocks.  Runs on CPU (a few seconds of oracle work)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["value"] > 0 and d["unit"] == "DOF-updates/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] >= 3 and d["n_gpus"] == 1 and d["dtype"] == "f64"
    assert d["config"]["dof"] == 4 * 64 ** 3 * 6 ** 3 and "workload" in d["config"]
    assert "model" not in d["config"]  # the workload is named, not a model
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_traffic_is_reported_only_for_the_captured_kernel_sources(monkeypatch):
    """roofline.traffic comes from an ncu capture of given kernel sources: the bench reports it
    only while the sources are those (digest), and never for a reduced problem."""
    sys.path.insert(0, ROOT)
    import bench
    digest = bench.kernel_sources_sha1()
    assert len(digest) == 40
    monkeypatch.setattr(bench, "TRAFFIC_SOURCES_SHA1", digest)
    assert bench.traffic_per_launch("euler3d", "f64", False) == bench.TRAFFIC_PER_LAUNCH[("euler3d", "f64")]
    assert bench.traffic_per_launch("euler3d", "f64", True) is None
    assert bench.traffic_per_launch("adv2d", "f64", False) is None
    monkeypatch.setattr(bench, "TRAFFIC_SOURCES_SHA1", "0" * 40)
    assert bench.traffic_per_launch("euler3d", "f32", False) is None


def test_committed_traffic_capture_is_of_the_committed_kernel_sources():
    """The DRAM traffic figures in bench.py were captured from the kernel sources as committed
    (their code digest), and the profile summary that records the capture names the same digest
    and the same per-launch figures; a kernel change without a new capture fails here."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.kernel_sources_sha1() == bench.TRAFFIC_SOURCES_SHA1
    summary = open(os.path.join(ROOT, "profiles", "stage_kernel_euler3d_deg5_64cubed.md")).read()
    assert bench.TRAFFIC_SOURCES_SHA1 in summary
    for dtype in ("f64", "f32"):
        figure = ("(%.4e)" % bench.TRAFFIC_PER_LAUNCH[("euler3d", dtype)]).replace("e+09", "e9")
        assert figure in summary
