"""Accuracy of the FP32 pooling geometry against long double (host build of the device header).

The pooling kernels form r^2, 1/r, the unit vector, t = 2r/rc - 1 and w = 1 - r/rc in FP32
with error-free transformations instead of FP64.  tests/geometry_check.cpp includes the
kernels' own header (pool_geometry.cuh) in its host mode, where every operation is one
rounded float operation as on the device, seeds 1/r with the correctly rounded value moved
by up to 2 ulp (the device's rsqrtf is approximate), and compares a million positions per
region with long-double values: next to the centre (r = 1e-6 .. 1e-2), in the bulk of the
ball, next to the cutoff (r = rc (1 - 1e-7 .. 1e-2)) and on the coordinate axes and planes.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def report(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("geo") / "geometry_check")
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-o", exe,
                    os.path.join(HERE, "geometry_check.cpp")], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    rows = {}
    for line in out.strip().splitlines():
        f = line.split()
        rows[f[0]] = dict(n=int(f[1]), ir=float(f[2]), unit=float(f[3]), t_ulp=float(f[4]), t_abs=float(f[5]),
                          w_rel=float(f[6]), w_abs=float(f[7]))
    return rows


@pytest.mark.parametrize("region", ["centre", "bulk", "cutoff", "axes"])
def test_geometry_accuracy(report, region):
    r = report[region]
    assert r["n"] > 900_000
    assert r["ir"] <= 0.5 + 1e-3          # 1/r correctly rounded
    assert r["unit"] <= 0.5 + 1e-3        # each unit-vector component correctly rounded
    assert r["t_ulp"] <= 1.5 and r["t_abs"] <= 3.0e-8   # 2r/rc - 1: within half an ulp of 1
    assert r["w_rel"] <= 2.5e-7           # 1 - r/rc keeps its relative accuracy up to the cutoff
