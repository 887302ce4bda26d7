"""Pins of the oracle's fast decoupled iterations: B' and B'' against an
independent complex Y-bus (tests/oracle_pins.ybus_matrix) of suitably
simplified networks, and the fixed point against the dense Newton solution."""
import numpy as np

import gridgen
import oracle
from tests import oracle_pins as pins


def test_matrices_are_imaginary_parts_of_ybus():
    sys = gridgen.synthetic_grid(60, 4, xfmr_frac=0.3, shift_frac=0.3, end_g_frac=0.2, cluster=20)
    sys.br_status[::11] = 0
    B1, B2, ns, pq = oracle.fdlf_matrices(sys)
    # B'': -Im(Y) of the network with its phase shifts removed
    s2 = sys.copy()
    s2.br_shift = np.zeros_like(sys.br_shift)
    Y = pins.ybus_matrix(s2)
    assert np.allclose(B2, -Y.imag[np.ix_(pq, pq)], rtol=1e-13, atol=1e-12)
    # B': -Im(Y) of a network of pure reactances (no resistance, charging, taps, shifts, shunts)
    s1 = sys.copy()
    s1.br_r = np.zeros_like(sys.br_r)
    s1.br_b = np.zeros_like(sys.br_b)
    s1.br_tap = np.ones_like(sys.br_tap)
    s1.br_shift = np.zeros_like(sys.br_shift)
    s1.br_g_fr = np.zeros_like(sys.br_g_fr)
    s1.br_g_to = np.zeros_like(sys.br_g_to)
    s1.sh_b = np.zeros_like(sys.sh_b)
    s1.sh_g = np.zeros_like(sys.sh_g)
    Y1 = pins.ybus_matrix(s1)
    assert np.allclose(B1, -Y1.imag[np.ix_(ns, ns)], rtol=1e-13, atol=1e-12)
    assert np.allclose(B1, B1.T) and np.allclose(B2, B2.T)


def test_fdlf_converges_to_the_newton_solution():
    sys = gridgen.grid_200()
    x0 = gridgen.flat_state(sys)
    xn, hn = oracle.newton_dense(sys, x0)
    xf, hf = oracle.fdlf(sys, x0)
    assert hf[-1] <= 1e-10 and hn[-1] <= 1e-10
    assert len(hf) > len(hn)                   # linear, not quadratic, convergence
    assert np.max(np.abs(xf - xn)) <= 1e-9
