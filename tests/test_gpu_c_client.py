"""The C ABI used from plain C: tests/c_abi_client.c, compiled with gcc against include/pf.h
and linked to libpf.so alone, evaluates the two-bus case through pf_residual_jacobian_host.
F is checked against its closed form, J against the oracle."""
import math
import os
import subprocess

import numpy as np
import pytest

import gridgen
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2011_11880_gb300")


@pytest.mark.gpu
def test_c_client_two_bus(tmp_path):
    import __graft_entry__
    __graft_entry__.build()
    exe = tmp_path / "c_abi_client"
    subprocess.run(["gcc", "-std=c99", "-O2", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c_abi_client.c"), "-o", str(exe), "-L", PKG, "-lpf",
                    "-Wl,-rpath," + PKG], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    vals = {ln.split()[0]: ln.split()[1:] for ln in out if ln}
    F = np.array([float(v) for v in vals["F"]])
    J = np.array([float(v) for v in vals["J"]])
    # closed form of the two-bus case (slack V = 1, theta = 0; line r = 0, x; PQ load P + jQ)
    x, p, q, th, v = 0.1, 0.5, 0.2, -0.05, 0.97
    assert F[0] == pytest.approx(v / x * math.sin(th) + p, rel=1e-12, abs=1e-10)
    assert F[1] == pytest.approx((v * v - v * math.cos(th)) / x + q, rel=1e-12, abs=1e-10)
    sys = gridgen.PowerSystem.build(2, branches=[(0, 1, 0.0, x, 0.0)], loads=[(1, p, q)], slack=(0, 1.0, 0.0))
    rp, ci, jv = oracle.jacobian(sys, np.array([0.0, th, 1.0, v]), oracle.REDUCED)
    assert [int(t) for t in vals["rowptr"]] == list(rp) and [int(t) for t in vals["colind"]] == list(ci)
    np.testing.assert_allclose(J, jv, rtol=1e-12, atol=1e-10)
