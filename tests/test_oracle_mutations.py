"""The oracle pins must catch plausible mistakes.

Each case copies ``oracle/pf_oracle.py`` into a temporary module with one
planted mistake (a dropped term, a wrong sign, a transposed operand, a wrong
exponent) and checks that at least one pin of ``oracle_pins`` rejects it.
The mistakes are planted in the CPU oracle only.
"""
import importlib.util
import os
import sys

import numpy as np
import pytest

import gridgen
from oracle import REDUCED, EXTENDED
from tests import oracle_pins as pins

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "pf_oracle.py")

MUTATIONS = [
    # (description, original text, mutated text)
    ("drop charging in Q_f", "qf = -vf * vf * (b + b_c / 2) / (tau * tau)", "qf = -vf * vf * (b) / (tau * tau)"),
    ("tap squared -> tap in P_f", "pf = vf * vf * (g + sys.br_g_fr) / (tau * tau)", "pf = vf * vf * (g + sys.br_g_fr) / (tau)"),
    ("sign of b sin in P_t", "pt = vt * vt * (g + sys.br_g_to) - vv * (g * cd - b * sd)", "pt = vt * vt * (g + sys.br_g_to) - vv * (g * cd + b * sd)"),
    ("phase shift sign", "delta = theta[f] - theta[t] - sys.br_shift\n    cd, sd = np.cos(delta), np.sin(delta)\n    vf, vt = V[f], V[t]\n    vv = vf * vt / tau\n    pf =",
     "delta = theta[f] - theta[t] + sys.br_shift\n    cd, sd = np.cos(delta), np.sin(delta)\n    vf, vt = V[f], V[t]\n    vv = vf * vt / tau\n    pf ="),
    ("end conductance on wrong end", "pt = vt * vt * (g + sys.br_g_to)", "pt = vt * vt * (g + sys.br_g_fr)"),
    ("transposed flow scatter", "np.add.at(fp, sys.br_to, pt)", "np.add.at(fp, sys.br_from, pt)"),
    ("shunt sign in Q", "np.add.at(fq, sys.sh_bus, -sys.sh_b * vs * vs)", "np.add.at(fq, sys.sh_bus, sys.sh_b * vs * vs)"),
    ("series b sign", "return r / d, -x / d", "return r / d, x / d"),
    ("Jacobian dQf/dVf missing factor 2", "d[\"Qf_Vf\"] = -2 * vf * (b + bc2)", "d[\"Qf_Vf\"] = -1 * vf * (b + bc2)"),
    ("Jacobian dPt/dtht sign", "d[\"Pt_tht\"] = -vv * (g * sd + b * cd)", "d[\"Pt_tht\"] = vv * (g * sd + b * cd)"),
    ("Jacobian dPf/dVt uses vt", "d[\"Pf_Vt\"] = -(vf / tau)", "d[\"Pf_Vt\"] = -(vt / tau)"),
    ("reduced: Q rows for PV buses", "pq = [b for b in range(n) if self.bus_type[b] == 0]", "pq = [b for b in range(n) if self.bus_type[b] != 2]"),
    ("pattern: drop diagonal entries", "            put(rmap[allb], cmap[allb], zero)", "            pass"),
]


def load_mutant(i, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation target not found: {old!r}"
    src = src.replace(old, new, 1)
    name = f"_oracle_mutant_{i}"
    spec = importlib.util.spec_from_loader(name, loader=None)
    mod = importlib.util.module_from_spec(spec)
    exec(compile(src, name, "exec"), mod.__dict__)
    sys.modules.pop(name, None)
    return mod


def run_all_pins(orc):
    s3 = gridgen.PowerSystem.build(
        4,                      # bus 3 is isolated: only its diagonal entries exist
        branches=[(0, 1, 0.01, 0.08, 0.04), (1, 2, 0.02, 0.12, 0.03, 1.0, 0.0, 0.002, 0.003),
                  (2, 0, 0.015, 0.10, 0.0, 0.97, 0.05), (1, 0, 0.012, 0.09, 0.02)],
        loads=[(1, 0.9, 0.3), (2, 0.5, 0.2), (3, 0.1, 0.05)], pvs=[(2, 0.6, 1.02)], slack=(0, 1.01, 0.05),
        shunts=[(1, 0.001, 0.15)])
    s = gridgen.synthetic_grid(24, 3, n_branch=32, end_g_frac=0.3, xfmr_frac=0.4, shift_frac=0.5, cluster=8)
    for sysm in (s3, s):
        pins.check_dimensions(orc, sysm)
        x = gridgen.perturbed_state(sysm, 2)
        pins.check_ybus(orc, sysm, x)
        pins.check_ohmic(orc, sysm, x)
        for mode in (REDUCED, EXTENDED):
            xe = gridgen.perturbed_state(sysm, 2, mode == EXTENDED)
            pins.check_jacobian_complex_step(orc, sysm, xe, mode)
            pins.check_pattern(orc, sysm, mode)


def test_unmutated_oracle_passes_all_pins():
    run_all_pins(load_mutant(-1, "import numpy as np", "import numpy as np"))


@pytest.mark.parametrize("i", range(len(MUTATIONS)), ids=[m[0] for m in MUTATIONS])
def test_pins_catch_mutation(i):
    desc, old, new = MUTATIONS[i]
    mod = load_mutant(i, old, new)
    with pytest.raises(AssertionError):
        run_all_pins(mod)
