"""Host logic of bench.py's roofline line (no GPU): the dominant kernel, the
achieved rate and fraction from CUDA-event times, and the DRAM traffic per
launch scaled from an ncu capture.

* every entry of bench.TRAFFIC_PER_WALKER names a summary under profiles/
  whose dram__bytes_read.sum + dram__bytes_write.sum, over the walkers of
  that capture, is the entry's bytes per walker (so an entry cannot drift
  from the evidence it cites);
* roofline() picks the kernel with the most event time, divides its
  algorithmic flops by the average launch time, and scales the traffic by
  the walker count;
* the tensor-core Green kernel reports no traffic (no capture of it feeds the
  table), and a kernel without a flop model reports no rate.
"""
import importlib
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
UNIT = {"KB": 1e3, "MB": 1e6, "GB": 1e9}


@pytest.fixture(scope="module")
def bench():
    return importlib.import_module("bench")


def _dram_bytes(path):
    """read + write bytes from a summary's dram__bytes rows: either one row
    'read / write' or a read row and a write row."""
    rows = [line for line in open(path) if line.startswith("| dram__bytes_")]
    assert rows, f"no dram__bytes rows in {path}"
    vals = [[float(v) * UNIT[u] for v, u in re.findall(r"([0-9.]+) (KB|MB|GB)", r.split("|")[2])] for r in rows]
    if len(vals[0]) >= 2:
        return vals[0][0] + vals[0][1]
    return vals[0][0] + vals[1][0]


def test_traffic_table_matches_profiles(bench):
    assert bench.TRAFFIC_PER_WALKER
    for key, (per_walker, summary, walkers) in bench.TRAFFIC_PER_WALKER.items():
        path = os.path.join(ROOT, summary)
        assert os.path.exists(path), f"{key}: {summary} is missing"
        assert f"_w{walkers}." in summary, f"{key}: capture walkers {walkers} not in the file name"
        measured = _dram_bytes(path)
        assert abs(per_walker * walkers - measured) <= 0.005 * measured, (key, per_walker * walkers, measured)


def test_roofline_arithmetic(bench):
    M, W = 257, 1024
    prof = {"green": {"ms": 49.3, "n_timed": 5}, "chain": {"ms": 34.3, "n_timed": 30},
            "tinv": {"ms": 22.8, "n_timed": 1}, "border": {"ms": 14.1, "n_timed": 30},
            "fields": {"ms": 0.0, "n_timed": 0}}
    r = bench.roofline(prof, M, W, "mixed")
    assert r["kernel"] == "green"
    avg_s = 49.3 / 5 / 1e3
    flops = (8.0 / 3.0 + 8.0) * M ** 3 * W
    assert r["avg_launch_ms"] == pytest.approx(avg_s * 1e3)
    assert r["achieved"] == pytest.approx(flops / avg_s / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["share_of_step"] == pytest.approx(49.3 / (49.3 + 34.3 + 22.8 + 14.1))
    per_walker = bench.TRAFFIC_PER_WALKER[("mixed", "green")][0]
    assert r["traffic"] == pytest.approx(per_walker * W)
    assert "608 walkers" in r["traffic_source"] and f"{W} walkers" in r["traffic_source"]


def test_chain_dominant_uses_tensor_peak(bench):
    M, W = 257, 1024
    prof = {"chain": {"ms": 60.0, "n_timed": 30}, "green": {"ms": 49.0, "n_timed": 5}}
    r = bench.roofline(prof, M, W, "mixed")
    assert r["kernel"] == "chain" and r["bound"] == "tensor"
    assert r["achieved"] == pytest.approx(3 * 8.0 * M ** 3 * W / (60.0 / 30 / 1e3) / 1e12)
    assert r["traffic"] == pytest.approx(bench.TRAFFIC_PER_WALKER[("mixed", "chain")][0] * W)


def test_tensor_core_green_and_unmodelled_kernels(bench):
    M, W = 515, 152
    r = bench.roofline({"green": {"ms": 86.5, "n_timed": 5}}, M, W, "mixed", green_tc=True)
    assert r["bound"] == "tensor" and r["traffic"] is None
    assert r["achieved"] == pytest.approx(3 * 12.0 * M ** 3 * W / (86.5 / 5 / 1e3) / 1e12)
    r = bench.roofline({"border": {"ms": 14.1, "n_timed": 30}}, 257, 1024, "mixed")
    assert r["kernel"] == "border" and r["achieved"] is None and r["frac"] is None
