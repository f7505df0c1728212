"""The FP64 reciprocal, reciprocal square root, quotient and square root that
the line search, the normalisation and the Gauss-Jordan pivots use on the GPU
(FP32 hardware seed, two Newton-Raphson steps; csrc/newton.cuh), against the
correctly rounded results.

Error bounds, in units in the last place of the correctly rounded result:
  recip  1 ulp: the second step leaves a relative error of about e^2 with
         e ~ 2^-46 after the first, so only the final rounding remains;
  div    2 ulps: the reciprocal's error plus the rounding of x * (1/y);
  rsqrt  2 ulps: the final product y (1.5 - h y) is rounded once, h = s y / 2
         carries one rounding, the seed's error is squared away twice;
  sqrt   3 ulps: s * rsqrt(s) adds one rounding to rsqrt's error.
Inputs sweep a logarithmic grid over 1e-35 .. 1e35 (both signs for the
reciprocal and quotient) with random mantissas, and the neighbours of the
1e-30 and 1e30 switch points, beyond which the IEEE operation is used."""
import ctypes
import math
import os
import subprocess
from decimal import Decimal, getcontext

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1105_5331_gb300", "csrc")


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    so = str(tmp_path_factory.mktemp("newton") / "newton_probe.so")
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-shared", "-Xcompiler", "-fPIC",
                    "-I", CSRC, os.path.join(HERE, "newton_probe.cu"), "-o", so], check=True)
    lib = ctypes.CDLL(so)
    lib.newton_probe.restype = ctypes.c_int
    return lib


def inputs():
    rng = np.random.default_rng(30)
    mags = 10.0 ** np.linspace(-35, 35, 3001) * rng.uniform(1.0, 10.0, 3001)
    edges = []
    for e in (1e-30, 1e30):
        v = e
        for _ in range(4):
            v = np.nextafter(v, 0.0)
        for _ in range(9):
            edges.append(v)
            v = np.nextafter(v, np.inf)
    x = np.concatenate([mags, -mags, np.array(edges), rng.uniform(0.5, 2.0, 2000)])
    y = rng.standard_normal(x.size) * 10.0 ** rng.uniform(-3, 3, x.size)
    return x, y


def ulps(got, exact):
    """|got - exact| in units in the last place of the double nearest exact."""
    ref = float(exact)
    ulp = math.ulp(ref)
    return float(abs(Decimal(got) - exact) / Decimal(ulp))


def test_newton_helpers_within_stated_ulps(probe):
    getcontext().prec = 60
    x, y = inputs()
    out = np.empty(4 * x.size)
    rc = probe.newton_probe(x.ctypes.data_as(ctypes.c_void_p), y.ctypes.data_as(ctypes.c_void_p), x.size,
                            out.ctypes.data_as(ctypes.c_void_p))
    assert rc == 0
    out = out.reshape(-1, 4)
    worst = {"recip": 0.0, "rsqrt": 0.0, "div": 0.0, "sqrt": 0.0}
    for i in range(x.size):
        X, Y = Decimal(float(x[i])), Decimal(float(y[i]))
        worst["recip"] = max(worst["recip"], ulps(out[i, 0], 1 / X))
        worst["div"] = max(worst["div"], ulps(out[i, 2], Y / X))
        if x[i] > 0:
            r = X.sqrt()
            worst["sqrt"] = max(worst["sqrt"], ulps(out[i, 3], r))
            worst["rsqrt"] = max(worst["rsqrt"], ulps(out[i, 1], 1 / r))
    print("worst ulps", worst)
    assert worst["recip"] <= 1.0 and worst["div"] <= 2.0
    assert worst["rsqrt"] <= 2.0 and worst["sqrt"] <= 3.0
