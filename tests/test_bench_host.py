"""Host logic of the benchmark's roofline (time-based, Sec. 3.4): the bound is
the larger of T_mem = bytes / HBM bandwidth and T_cmp = binding-pipe
instructions / pipe peak, and the fraction is that time over the measured
one, reported against the bound's own peak."""
import pytest

import bench


def _info(E, bytes_per_element, ops_per_element, pipe=1):
    return {"E": E, "bytes_per_element": bytes_per_element, "pipe_ops_per_element": ops_per_element,
            "flops_ax_per_element": 1000.0, "pipe": pipe}


def test_alu_bound():
    # 1e6 elements x 1e6 FP32-pipe lane-instructions at 128 x 152 lanes x 2 GHz = 25.7 ms
    info = _info(10 ** 6, 8.0, 1e6)
    peak = 128 * 152 * 2000e6
    r = bench._roofline(info, ms=50.0, sm_mhz=2000.0, hbm_gbs=6777.0)
    assert r["bound"] == "alu"
    assert r["peak"] == pytest.approx(peak / 1e12)
    assert r["frac"] == pytest.approx((1e12 / peak) / 50e-3)
    assert r["frac"] == pytest.approx(r["frac_time_roofline"])


def test_hbm_bound():
    info = _info(10 ** 6, 64e3, 1.0)
    r = bench._roofline(info, ms=20.0, sm_mhz=2000.0, hbm_gbs=6777.0)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(64e9 / 20e-3 / 1e9)
    assert r["frac"] == pytest.approx((64e9 / 6777e9) / 20e-3)
    assert r["frac"] == pytest.approx(r["frac_time_roofline"])


def test_fp64_pipe_peak():
    # native FP64 kernels are bound by the FP64 pipe: 2 FMA per SM per clock
    r = bench._roofline(_info(10 ** 5, 8.0, 1e4, pipe=0), ms=10.0, sm_mhz=2070.0, hbm_gbs=6777.0)
    assert r["bound"] == "alu" and r["peak"] == pytest.approx(2 * 152 * 2070e6 / 1e12)
