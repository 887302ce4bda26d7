"""Pins of the oracle's reactive-limit handling in the extended formulation
(Sec. II-A: the same formulation serves before and after a PV generator
switches to a PQ load; a generator held at a limit has g_V = Q_g - Q_lim).

The pins do not re-type the oracle's formulas: the Jacobian of the switched
rows is checked by complex-step differentiation of the residual, the pattern
by comparison across modes, and the switched solution against a different
formulation of the same physics -- the reduced formulation of a system in
which that generator bus is an ordinary PQ bus injecting (P_g, Q_lim)."""
import numpy as np

import gridgen
import oracle
from oracle import EXTENDED, REDUCED
from tests import oracle_pins as pins


def _modes(sys, seed):
    rng = np.random.default_rng(seed)
    ng = sys.n_pv + 1
    mode = rng.integers(0, 3, ng).astype(np.int8)
    qlim = rng.uniform(-0.5, 0.8, ng)
    return mode, qlim


def test_pattern_is_the_same_in_every_mode():
    sys = gridgen.grid_200()
    x = gridgen.perturbed_state(sys, 2, True)
    rp0, ci0, _ = oracle.jacobian(sys, x, EXTENDED)
    for seed in range(3):
        mode, _ = _modes(sys, seed)
        rp, ci, _ = oracle.jacobian(sys, x, EXTENDED, gen_mode=mode)
        assert np.array_equal(rp, rp0) and np.array_equal(ci, ci0)


def test_switched_jacobian_matches_complex_step():
    for sys in (gridgen.synthetic_grid(30, 7, n_branch=39, cluster=10), gridgen.grid_200()):
        mode, qlim = _modes(sys, 5)
        x = gridgen.perturbed_state(sys, 3, True)
        fm = oracle.Formulation(sys, EXTENDED)
        rp, ci, jv = oracle.jacobian(sys, x, EXTENDED, gen_mode=mode)
        J = oracle.csr_to_dense(rp, ci, jv, fm.n_cols)
        Jc = pins.complex_step_columns(
            lambda xc: oracle.residual(sys, xc, EXTENDED, gen_mode=mode, gen_qlim=qlim), x,
            pins.column_positions(sys, fm))
        pins.assert_close(J, Jc, 1e-12, 1e-11, "switched J vs complex step")
        # the held rows read Q_g - Q_lim
        F = oracle.residual(sys, x, EXTENDED, gen_mode=mode, gen_qlim=qlim)
        held = mode != 0
        n = sys.n_bus
        qg = x[2 * n:2 * n + sys.n_pv + 1]
        assert np.array_equal(F[fm.row_gv[held]], qg[held] - qlim[held])


def test_vjp_with_held_generators_matches_complex_step():
    sys = gridgen.synthetic_grid(30, 7, n_branch=39, cluster=10)
    mode, qlim = _modes(sys, 9)
    x = gridgen.perturbed_state(sys, 1, True)
    fm = oracle.Formulation(sys, EXTENDED)
    v = gridgen.gaussian_cotangents(fm.n_rows, 1)[0]
    g = oracle.vjp(sys, x, v, EXTENDED, gen_mode=mode)["x"]
    gc = pins.complex_step_columns(
        lambda xc: v @ oracle.residual(sys, xc, EXTENDED, gen_mode=mode, gen_qlim=qlim), x, range(x.shape[0]))
    pins.assert_close(g, gc, 1e-12, 1e-11, "v^T J with held generators")


def _as_pq(sys, i, q):
    """The system with PV unit i removed and its bus given (P_g, q) as a negative load."""
    s = sys.copy()
    keep = np.arange(sys.n_pv) != i
    b, p = int(sys.pv_bus[i]), float(sys.pv_p[i])
    s.pv_bus, s.pv_p, s.pv_vset = sys.pv_bus[keep], sys.pv_p[keep], sys.pv_vset[keep]
    s.load_bus = np.concatenate([sys.load_bus, [b]])
    s.load_p = np.concatenate([sys.load_p, [-p]])
    s.load_q = np.concatenate([sys.load_q, [-q]])
    return s


def test_held_generator_equals_pq_bus_in_the_reduced_formulation():
    sys = gridgen.grid_200()
    n = sys.n_bus
    xe, hist = oracle.newton_dense(sys, gridgen.flat_state(sys, True), EXTENDED)
    assert hist[-1] <= 1e-10
    ng = sys.n_pv + 1
    for i in (3, 17):
        q_star = 0.5 * xe[2 * n + i]                     # hold unit i at half its unconstrained output
        mode = np.zeros(ng, np.int8)
        qlim = np.zeros(ng)
        mode[i], qlim[i] = 1, q_star
        xh, hh = oracle.newton_dense(sys, xe, EXTENDED, gen_mode=mode, gen_qlim=qlim)
        assert hh[-1] <= 1e-10
        assert xh[2 * n + i] == q_star or abs(xh[2 * n + i] - q_star) <= 1e-12
        s_pq = _as_pq(sys, i, q_star)
        xr, hr = oracle.newton_dense(s_pq, xe[:2 * n].copy(), REDUCED)
        assert hr[-1] <= 1e-10
        # same network state; the bus of unit i now floats in voltage
        assert np.max(np.abs(xh[:2 * n] - xr)) <= 1e-9
        assert abs(xh[n + sys.pv_bus[i]] - sys.pv_vset[i]) > 1e-6


def test_newton_qlim_switches_and_respects_limits():
    sys = gridgen.grid_200()
    n = sys.n_bus
    ng = sys.n_pv + 1
    xe, _ = oracle.newton_dense(sys, gridgen.flat_state(sys, True), EXTENDED)
    q0 = xe[2 * n:2 * n + ng]
    q_max = np.full(ng, np.inf)
    q_min = np.full(ng, -np.inf)
    tight = np.array([2, 9, 21])
    q_max[tight] = q0[tight] - 0.05                       # these exceed their upper limit
    x, mode, qlim, rounds = oracle.newton_qlim(sys, gridgen.flat_state(sys, True), q_min, q_max)
    assert rounds >= 2
    qg = x[2 * n:2 * n + ng]
    assert set(np.nonzero(mode)[0]) >= set(tight.tolist())
    assert np.all(qg[mode == 1] == q_max[mode == 1]) or np.allclose(qg[mode == 1], q_max[mode == 1], atol=1e-12)
    assert np.all(qg[mode == 0] <= q_max[mode == 0] + 1e-9)
    assert np.max(np.abs(oracle.residual(sys, x, EXTENDED, gen_mode=mode, gen_qlim=qlim))) <= 1e-10
