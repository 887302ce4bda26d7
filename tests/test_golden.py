"""Golden fixtures: the paper's printed numbers (consistency) and the oracle's
regression record on the 200-bus case (written by tests/golden/make_golden.py
from the oracle only)."""
import hashlib
import json
import os

import numpy as np
import pytest

import gridgen
import oracle

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(HERE, name)) as fh:
        return json.load(fh)


def test_paper_tables_consistent():
    """Table IV row sums reproduce Table III equation times of workflows 1, 3 and 5
    (serial, threaded, SIMD intra-model) within the join overhead."""
    p = load("paper_numbers.json")
    t4 = p["table_IV_equation_us_by_model"]
    t3 = p["table_III_equation_jacobian_ms"]
    for row, wf in (("serial", "wf1"), ("threaded", "wf3"), ("simd", "wf5")):
        total_ms = sum(t4[row]) / 1000.0
        assert abs(total_ms - t3[wf][0]) <= 0.3 * t3[wf][0] + 0.05
    # the line model dominates the serial equation time (Sec. IV-C)
    assert t4["serial"][3] / sum(t4["serial"]) > 0.99


def sha(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


@pytest.mark.parametrize("mode,name", [(oracle.REDUCED, "reduced"), (oracle.EXTENDED, "extended")])
def test_oracle_regression_200(mode, name):
    g = load("oracle_200bus.json")["modes"][name]
    s = gridgen.grid_200()
    ext = mode == oracle.EXTENDED
    for k, rec in enumerate(g["states"]):
        x = gridgen.flat_state(s, ext) if k == 0 else gridgen.perturbed_state(s, k, ext)
        F = oracle.residual(s, x, mode)
        rp, ci, jv = oracle.jacobian(s, x, mode)
        if k == 0:
            assert F.shape[0] == g["n_rows"] and rp[-1] == g["nnz"]
            assert sha(rp.astype(np.int32)) == g["rowptr_sha256"]
            assert sha(ci.astype(np.int32)) == g["colind_sha256"]
        np.testing.assert_allclose(F[::17], rec["F_every_17th"], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(jv[::97], rec["J_every_97th"], rtol=1e-12, atol=1e-12)
