"""Host-side logic of bench.py on CPU: the JSON line of the reference arm (the
oracle on the host cores), the DRAM-traffic record that the roofline reads
(scaled by rails, withdrawn when the kernel source changes), and the parsing
of the clock samples taken during the timed region."""
import hashlib
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in line, k
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["steps"] == 1 and line["warmup"] == 3 and line["n_gpus"] == 1
    assert line["config"]["workload"] == "hysteresis_65536x1024"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"]
    assert cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def _traffic_fixture(tmp_path, source: bytes, recorded_sha: str):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "k.cu").write_bytes(source)
    rec = {"kernel_source": "k.cu", "kernel_source_sha256": recorded_sha, "rails": 16384,
           "steps_per_launch": 10000, "dram_bytes_read": 1000, "dram_bytes_write": 24}
    (tmp_path / "profiles" / "sweep_traffic.json").write_text(json.dumps(rec))


def test_traffic_scaled_by_rails_while_the_source_matches(tmp_path, monkeypatch):
    src = b"__global__ void k() {}\n"
    _traffic_fixture(tmp_path, src, hashlib.sha256(src).hexdigest())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic_per_launch(16384, 10000) == 1024
    assert bench._traffic_per_launch(65536, 10000) == 4096
    # a capture of launches of another length says nothing about this one
    assert bench._traffic_per_launch(65536, 1000) is None


def test_traffic_withdrawn_when_the_source_changed(tmp_path, monkeypatch):
    _traffic_fixture(tmp_path, b"changed\n", hashlib.sha256(b"original\n").hexdigest())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic_per_launch(65536, 10000) is None
    monkeypatch.setattr(bench, "ROOT", str(tmp_path / "missing"))
    assert bench._traffic_per_launch(65536, 10000) is None


def test_committed_traffic_record_names_the_sweep_kernel_source():
    with open(os.path.join(ROOT, "profiles", "sweep_traffic.json")) as f:
        rec = json.load(f)
    assert rec["kernel_source"] == "paper_2511_09413_gb300/csrc/kmc_sweep.cu"
    assert rec["rails"] > 0 and rec["dram_bytes_read"] > 0 and rec["dram_bytes_write"] >= 0
    assert rec["steps_per_launch"] > 0
    assert "--clock-control none" in rec["command"]


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass

    def join(self, timeout=None):
        pass


@pytest.mark.parametrize("lines,median,reasons", [
    (["2070, 2070, 900.1, Not Active, Not Active, Not Active, Not Active"] * 3, 2070.0, []),
    (["1980, 2070, 1390.0, Not Active, Not Active, Not Active, Active",
      "2010, 2070, 1395.2, Not Active, Not Active, Not Active, Active",
      "[N/A], 2070, 1.0, Not Active, Not Active, Not Active, Not Active",
      "short line"], 1995.0, ["sw_power_cap"]),
    (["1500, 2070, 700.0, Active, Not Active, Active, Not Active"], 1500.0,
     ["hw_slowdown", "sw_thermal_slowdown"]),
])
def test_clock_samples_parsed(lines, median, reasons):
    s = bench.ClockSampler(0)
    s.proc, s.thread, s.lines = _Done(), _Done(), list(lines)
    got = s.stop()
    assert got["sm_mhz"] == median
    assert got["sm_max_mhz"] == 2070.0
    assert got["reasons"] == reasons


def test_clock_sampler_without_nvidia_smi():
    s = bench.ClockSampler(0)
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_alu_peak_is_derived_from_unit_counts_and_clock():
    """The roofline's integer-pipe peak: 152 SMs x 64 IMAD lanes per clock at
    the maximum SM clock over 34 IMAD issue slots per Philox4x32-10 block
    (16 widening multiplies at two slots, two low halves at one)."""
    assert bench.PHILOX_IMAD_SLOTS == 16 * 2 + 2
    peak = bench.SMS * bench.IMAD_PER_SM_PER_CLK * 2070e6 / bench.PHILOX_IMAD_SLOTS
    assert abs(peak - 5.922e11) < 1e8
