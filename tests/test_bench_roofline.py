"""bench.py's roofline arithmetic, on CPU.

A kernel's roofline takes the slower of its two bounds: the algorithmic bytes
at the measured copy bandwidth, or its tensor work at the given tensor peak.
`achieved` is that algorithmic quantity divided by the measured time, `frac`
is achieved / peak, and `traffic` scales the per-row DRAM bytes of an ncu
capture to the launch's rows.  These checks fix the numbers every roofline
entry of the bench line is built from.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

PK = {"hbm": 6000.0, "bf16": 2000.0, "bf16_sustained": 1500.0, "kind": "measured"}


def test_hbm_bound_kernel():
    # 6 GB at 6,000 GB/s is 1 ms; 0.3 TFLOP at 1,500 TFLOP/s is 0.2 ms: HBM-bound
    r = bench.roofline("sketch", 2.0, 6e9, 0.3e12, 1500.0, PK, 1000, "no-such-workload")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(3000.0)  # 6 GB in 2 ms
    assert r["peak"] == 6000.0 and r["frac"] == pytest.approx(0.5)
    assert r["traffic"] is None and r["peak_kind"] == "measured"


def test_tensor_bound_kernel():
    # 3 TFLOP at 1,500 TFLOP/s is 2 ms, above the 1 ms of its 6 GB: tensor-bound
    r = bench.roofline("project", 4.0, 6e9, 3e12, 1500.0, PK, 1000, "no-such-workload")
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(750.0)  # 3 TFLOP in 4 ms
    assert r["frac"] == pytest.approx(0.5)
    assert r["flops_per_launch"] == 3e12 and r["bytes_per_launch"] == 6e9


def test_no_tensor_work_is_hbm_bound():
    r = bench.roofline("chain_main", 1.0, 6e9, 0, 1.0, PK, 10, "no-such-workload")
    assert r["bound"] == "hbm" and r["frac"] == pytest.approx(1.0)


def test_traffic_scales_the_captured_bytes_per_row():
    key = next(iter(bench.TRAFFIC_PER_ROW))
    per_row = bench.TRAFFIC_PER_ROW[key]
    r = bench.roofline(key[1], 1.0, 1e9, 0, 1.0, PK, 12345, key[0])
    assert r["traffic"] == pytest.approx(per_row * 12345)


def test_captured_traffic_matches_the_algorithmic_bytes():
    # the ncu captures of the headline kernels read X once: DRAM bytes per row
    # within 1 % of n + k (sketch, pass F) and n + 4k (reduction map)
    n, k = 4096, 256
    want = {"sketch": n + k, "chain_main": n + k, "project": n + 4 * k}
    for (workload, kern), per_row in bench.TRAFFIC_PER_ROW.items():
        if workload.startswith("e4m3_binary") and kern in want:
            assert per_row == pytest.approx(want[kern], rel=0.01), (workload, kern)
