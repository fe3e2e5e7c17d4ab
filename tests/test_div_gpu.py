"""The step kernels' division for normal positive operands (lbm_math.cuh:
the hardware reciprocal approximation, one Newton-Raphson step and
Markstein's residual correction) against the IEEE division, bit for bit, on
seeded operand pairs log-uniform over [2^-10, 2^10] with either sign of the
dividend (a superset of the closure's phi-hat / (1 - mdot / 2) and the
reciprocals of rho and tau_f)."""
import ctypes
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2403_16122_gb300", "csrc")


def test_div_normal_equals_ieee_division(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    lib = str(tmp_path / "libdivcheck.so")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "-shared", "-Xcompiler", "-fPIC", f"-I{CSRC}",
                    os.path.join(HERE, "div_check.cu"), "-o", lib], check=True)
    f = ctypes.CDLL(lib).div_check
    f.argtypes = [ctypes.c_longlong, ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_ulonglong),
                  ctypes.POINTER(ctypes.c_uint)]
    bad, ulp = ctypes.c_ulonglong(0), ctypes.c_uint(0)
    n = 1 << 26
    assert f(n, 20240324, ctypes.byref(bad), ctypes.byref(ulp)) == 0
    print(f"{n} pairs: {bad.value} differ from the IEEE quotient (max {ulp.value} ulp)")
    assert bad.value == 0
