"""The benchmark's roofline arithmetic, on CPU: the algorithmic bytes per
particle-step of the 3D RK4 workload with three properties and 20 particles
per cell, and the roofline object built from them (achieved = bytes x
particles / launch time; frac = achieved / peak)."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_algorithmic_bytes(bench):
    # state: x 24 + x-hat 24 + id 8 + props 24 = 80 B, read and written
    # (160), the new-cell key (8), cell data (8 nodes x 3 components x 8 B +
    # one vertex 24 B + a 4 B offset) / 20
    assert bench.step_bytes(3, 3, 20) == pytest.approx(160 + 8 + (192 + 24 + 4) / 20)
    assert round(bench.step_bytes(3, 3, 20)) == 179
    # the advect kernel's share: the cell u32 read and written instead of
    # the key, no offset
    assert bench.advect_bytes(3, 20, 3) == pytest.approx(2 * (24 + 24 + 4 + 8 + 24) + (192 + 24) / 20)
    assert bench.advect_bytes(3, 20, 3) == pytest.approx(178.8)
    # FP32-basis form: x-hat and the nodal values at 4 B
    assert bench.advect_bytes(3, 20, 3, 4, 4) == pytest.approx(150.0)


def test_roofline_object(bench):
    r = bench.roofline_object(0, 10.0, 1.0e9, 178.8, 7000.0)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(178.8 * 1.0e9 / 0.010 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 7000.0)
    # the DRAM traffic of one launch scales the captured bytes per particle
    assert r["traffic"] == pytest.approx(bench.ADVECT_DRAM_BYTES_PER_PARTICLE[0] * 1.0e9)
