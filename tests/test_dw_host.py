"""Host check of the double-word arithmetic (csrc/dw.cuh) that the FP64-accurate
AxLocal kernels run on the FP32 pipe.

The header is compiled for the CPU with stand-ins for its CUDA intrinsics (each
the correctly rounded IEEE operation it names, tests/dw_host/cuda_runtime.h)
and every building block is compared with long-double references on seeded
random operands spanning 2^-20..2^20.  Errors are in units of 2^-47 times the
magnitudes involved; the bounds follow the published ones (TwoSum error-free;
DW x DW within 4u^2 = 2 units, Joldes-Muller-Popescu 2017) with small
multiples for the compound operations.  The AxLocal tolerance of 1e-12
relative is about 2^-40 = 128 units, so a kernel that chains a few dozen of
these operations per output stays inside it.  This checks the arithmetic, not
the kernels (the GPU parity tests do that).
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
BOUNDS = {"two_sum": 0.0, "add": 2.0, "mul": 2.0, "fma": 4.0, "mac": 8.0, "acc_sum": 8.0, "lazy": 8.0,
          "div": 8.0, "conv": 0.5, "sum3": 4.0, "conv_direct": 0.5, "sum3_direct": 4.0, "bad_direct": 0.0}


def test_double_word_building_blocks(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "dw_check")
    src = os.path.join(HERE, "dw_host", "dw_check.cpp")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", os.path.join(HERE, "dw_host"), "-o", exe,
                    src], check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    errs = {k: float(v) for k, v in (line.split() for line in out.strip().splitlines())}
    assert set(errs) == set(BOUNDS)
    for k, bound in BOUNDS.items():
        assert errs[k] <= bound, (k, errs[k], bound)
