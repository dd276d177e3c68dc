"""bench.py's roofline entry (host logic, no GPU): the achieved rate is 12 FLOP per cell
over the launch time, the FP32 peak is 2 x 128 lanes x SMs x clock, and the DRAM traffic
comes from profiles/forward_traffic.json only for the exact kernel and cell count a
capture covered."""
import json
import os

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INFO = {"sms": 152, "max_clock_mhz": 2070.0}


def _traffic_table():
    return json.load(open(os.path.join(ROOT, "profiles", "forward_traffic.json")))


def test_roofline_arithmetic(monkeypatch):
    monkeypatch.setattr(bench, "_peaks", lambda: {"sm_max_mhz": 2070.0})
    dom = {"kernel": "k_unprofiled", "cells": 10**12, "ms": 1000.0, "branch": "x"}
    r = bench.roofline(dom, INFO)
    peak = 2.0 * 128 * 152 * 2070e6 / 1e12
    assert r["peak"] == pytest.approx(peak)
    assert r["achieved"] == pytest.approx(12.0 * 1e12 / 1.0 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / peak)
    assert r["traffic"] is None  # no capture for this kernel
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"


@pytest.mark.parametrize("kernel", sorted(_traffic_table()))
def test_traffic_only_for_the_captured_launch(monkeypatch, kernel):
    monkeypatch.setattr(bench, "_peaks", lambda: {})
    for cells, ent in _traffic_table()[kernel].items():
        dom = {"kernel": kernel, "cells": int(cells), "ms": 1.0, "branch": "x"}
        assert bench.roofline(dom, INFO)["traffic"] == ent["bytes_per_launch"]
        # another workload of the same kernel has no measured traffic
        dom["cells"] = int(cells) + 1
        assert bench.roofline(dom, INFO)["traffic"] is None


def test_traffic_table_names_kernels_the_library_reports():
    from paper_2606_25738_gb300 import phmm
    names = set(phmm.SHORT_KERNELS) | set(phmm.PACKED_KERNELS) | set(phmm.LONG_KERNELS)
    for kernel in _traffic_table():
        assert kernel in names, kernel
