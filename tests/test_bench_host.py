"""Host-side pieces of bench.py: the roofline object's arithmetic, the
measured-traffic lookup (reported only while the kernel source is the one
the ncu capture was taken from) and the timing defaults."""
import hashlib
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _Wl:
    w = 300


def test_timing_defaults(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert a.gpus == 1 and a.warmup >= 3 and a.steps >= 1 and a.impl == "momenti"


def test_measured_traffic_follows_the_source():
    for kernel, (path, sha, nbytes) in bench.NCU_TRAFFIC.items():
        with open(os.path.join(ROOT, path), "rb") as fh:
            same = hashlib.sha256(fh.read()).hexdigest() == sha
        assert bench.measured_traffic(kernel) == (nbytes if same else None)
    assert bench.measured_traffic("no_such_kernel") is None


def test_roofline_arithmetic():
    pk = {"hbm_gbs": 6779.0, "tflops": 1933.3, "tflops_sustained": 1727.1,
          "sm_max_mhz": 2070.0, "src": "measured"}
    info = {"M": 99701, "D": 8, "L": 200, "K": 8}
    st = {"n_candidates": 1000}
    steps, ms = 5, 5 * 44.0
    r = bench.roofline("allpairs", ms, steps, info, st, _Wl, steps, pk)
    excl = _Wl.w // 2
    pairs = (info["M"] - excl - 1) * (info["M"] - excl) / 2.0
    work = 8.0 * info["D"] * pairs          # the minimal flop count per pair and dim
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(work * steps / (ms / 1e3) / 1e12)
    assert r["peak"] == pytest.approx(152 * 128 * 2 * 2070.0 * 1e6 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["ms_per_launch"] == pytest.approx(44.0)
    t = bench.roofline("proj_hash_tc", 5 * 2.9, steps, info, st, _Wl, steps, pk)
    assert t["bound"] == "tensor" and t["peak"] == pk["tflops_sustained"]
    assert t["achieved"] == pytest.approx(2.0 * 99701 * 8 * 200 * 8 * 300 / 2.9e-3 / 1e12)
    assert bench.roofline("allpairs", 0.0, 0, info, st, _Wl, steps, pk) is None


def test_clock_samples_parse():
    rows = "\n".join([
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2040, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2055, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ])
    c = bench.Clocks.parse(rows)
    assert c == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    hot = bench.Clocks.parse("0, 1500, 2070, 1400, 0x8, Not Active, Active, Not Active, Not Active")
    assert hot["reasons"] == ["hw_thermal_slowdown"]
    assert bench.Clocks.parse("") == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_clock_sampler_end_to_end(tmp_path, monkeypatch):
    # a stand-in nvidia-smi on PATH: the sampler starts it, stops it and
    # parses what it wrote
    import time
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\n"
                    "echo '0, 2070, 2070, 800, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "echo '0, 2060, 2070, 900, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "exec sleep 30\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}:{os.environ['PATH']}")
    c = bench.Clocks(0)
    c.start()
    time.sleep(1.0)
    out = c.stop()
    assert out == {"sm_mhz": 2065.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 2}


def test_collision_roofline_arithmetic():
    # 12 B per index entry per (level, repetition) processed plus 16 D B per
    # compared bucket pair, over the summed time of the collision kernels
    pk = {"hbm_gbs": 6779.0, "tflops": 1933.3, "tflops_sustained": 1727.1,
          "sm_max_mhz": 2070.0, "src": "measured"}
    info = {"M": 99701, "D": 8, "L": 200, "K": 8}
    assert bench.reps_processed({"stop_i": 0, "stop_j": 0, "switch_level": 1}, 8, 200) == 7 * 200 + 1
    assert bench.reps_processed({"stop_i": 3, "stop_j": 17, "switch_level": 0}, 8, 200) == 5 * 200 + 17
    assert bench.reps_processed({"stop_i": 0, "stop_j": 0, "switch_level": 0}, 8, 200) == 8 * 200
    st = {"stop_i": 0, "stop_j": 0, "switch_level": 1, "n_pair_checks": 10 ** 9}
    r = bench.roofline("collision", 20.0, 300, info, st, _Wl, 1, pk)
    work = 12.0 * 99701 * 8 * 1401 + 16.0 * 8 * 1e9
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(work / 0.020 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6779.0)
