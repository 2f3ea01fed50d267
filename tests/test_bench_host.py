"""Host logic of bench.py that needs no GPU: the clock sampler's parsing
(the throttle reasons decide whether a run is kept) and the JSON line of the
reference arm at N = 1."""
import json
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_samples_and_throttle_reasons():
    import bench
    c = bench.Clocks()
    fd, c.path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as f:
        f.write("0, 2070, 2070, 812.3, 0x0000000000000000, Not Active, Not Active, "
                "Not Active, Not Active\n")
        f.write("0, 1980, 2070, 1399.0, 0x0000000000000004, Not Active, Not Active, "
                "Not Active, Active\n")
        f.write("0, [N/A], 2070, 10.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("a line nvidia-smi did not finish\n")
    c.proc = _FakeProc()
    d = c.stop()
    assert d["samples"] == 2
    assert d["sm_mhz"] == 2025.0 and d["sm_max_mhz"] == 2070.0 and d["power_w_max"] == 1399.0
    assert d["reasons"] == ["sw_power_cap"]  # kept and noted; no slowdown reason
    assert not os.path.exists(c.path)


def test_clocks_without_nvidia_smi():
    import bench
    c = bench.Clocks()
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]


@pytest.mark.timeout(300)
def test_reference_arm_line_carries_every_key():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=280)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["ms_per_step"] == pytest.approx(1e3 / d["value"])
    assert d["config"]["workload"].startswith("block100")
    assert "extrapolated" in d["config"]["workload"] and d["config"]["nnz"] == 376_541_249
    assert d["config"]["pcg_iters_scaled_to"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"]
    assert "4x33x4" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_ap_roofline_figures():
    """The A.p line: algorithmic bytes per launch over the mean event time,
    against the measured copy bandwidth; nothing when nothing was timed."""
    import bench
    pr = {"total_ms": 3.5, "launches": 20, "bytes_per_launch": 689588680.0}
    d = bench.ap_roofline(pr, 0)
    assert d["form"] == "FP64" and d["launches"] == 20
    assert d["avg_launch_ms"] == pytest.approx(0.175)
    assert d["achieved"] == pytest.approx(689588680.0 / 0.175e-3 / 1e9)
    assert d["frac"] == pytest.approx(d["achieved"] / bench.hbm_peak())
    assert bench.ap_roofline(pr, 1)["form"].startswith("float-float")
    assert bench.ap_roofline(None, 0) is None
    assert bench.ap_roofline({"total_ms": 0.0, "launches": 0, "bytes_per_launch": 1.0}, 0) is None


def test_default_run_stays_short():
    """The default serving legs (what the driver's run includes) are the
    24-request trace with the streams and plain FP64 arms; the larger
    traces and other arms take flags."""
    import bench
    old = sys.argv
    try:
        sys.argv = ["bench.py"]
        a = bench.parse()
    finally:
        sys.argv = old
    assert a.serve_requests == 24 and a.serve_instances == 24
    assert a.serve_arms.split(",") == ["batched_streams", "plain_fp64"]
    assert all(n in bench.SERVE_ARMS for n in a.serve_arms.split(","))
    assert a.ap_split == 0 and not a.serve_only
