"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Sec. II-B Eq. (4) (active power at the line terminals), Sec. II-A (models
and extended formulation, Eqs. 1-3), and the closed forms / identities
listed in ``oracle_pins``.  CPU only.
"""
import numpy as np
import pytest

import gridgen
import oracle
from oracle import REDUCED, EXTENDED
from tests import oracle_pins as pins


def three_bus():
    """Triangle with a parallel branch, a tapped phase-shifting transformer,
    end conductances, a shunt, one out-of-service branch, a PV and a load."""
    return gridgen.PowerSystem.build(
        3,
        branches=[
            (0, 1, 0.01, 0.08, 0.04),
            (1, 2, 0.02, 0.12, 0.03, 1.0, 0.0, 0.002, 0.003),
            (2, 0, 0.015, 0.10, 0.0, 0.97, 0.05),
            (1, 0, 0.012, 0.09, 0.02),           # parallel to branch 0, reversed
            (0, 2, 0.03, 0.2, 0.0, 1.0, 0.0, 0.0, 0.0, 0),   # out of service
        ],
        loads=[(1, 0.9, 0.3), (2, 0.5, 0.2)],
        pvs=[(2, 0.6, 1.02)],
        slack=(0, 1.01, 0.05),
        shunts=[(1, 0.001, 0.15)],
    )


def small_grid(seed=7, n=30, **kw):
    return gridgen.synthetic_grid(n, seed, n_branch=int(1.3 * n), end_g_frac=0.2,
                                  xfmr_frac=0.3, shift_frac=0.3, cluster=10, **kw)


STATES = [0, 1, 2]


def state(sys, k, mode=REDUCED):
    ext = mode == EXTENDED
    return gridgen.flat_state(sys, ext) if k == 0 else gridgen.perturbed_state(sys, k, ext)


# --- Eq. (4) ---------------------------------------------------------------

def test_eq4_active_power_reduction():
    """With tau = 1, phi = 0 the oracle's P_f, P_t are Eq. (4) of Sec. II-B."""
    s = small_grid()
    s.br_tap[:] = 1.0
    s.br_shift[:] = 0.0
    x = gridgen.perturbed_state(s, 3)
    n = s.n_bus
    th, v = x[:n], x[n:]
    pf, _, pt, _ = oracle.branch_flows(s, th, v)
    h, k = s.br_from, s.br_to
    gl = s.br_r / (s.br_r ** 2 + s.br_x ** 2)
    bl = -s.br_x / (s.br_r ** 2 + s.br_x ** 2)
    thk = th[h] - th[k]
    ph = v[h] ** 2 * (gl + s.br_g_fr) - v[h] * v[k] * (gl * np.cos(thk) + bl * np.sin(thk))
    pk = v[k] ** 2 * (gl + s.br_g_to) - v[h] * v[k] * (gl * np.cos(thk) - bl * np.sin(thk))
    pins.assert_close(pf, ph, what="P_h")
    pins.assert_close(pt, pk, what="P_k")


# --- independent complex formulations ----------------------------------------

@pytest.mark.parametrize("k", STATES)
def test_mismatch_matches_ybus_three_bus(k):
    s = three_bus()
    pins.check_ybus(oracle, s, state(s, k))


@pytest.mark.parametrize("k", STATES)
def test_mismatch_matches_ybus_random(k):
    s = small_grid()
    pins.check_ybus(oracle, s, state(s, k))


def test_mismatch_matches_ybus_200():
    s = gridgen.grid_200()
    pins.check_ybus(oracle, s, state(s, 4))


@pytest.mark.parametrize("k", STATES)
def test_branch_losses_ohm(k):
    for s in (three_bus(), small_grid()):
        pins.check_ohmic(oracle, s, state(s, k))


# --- hand-derived closed forms -------------------------------------------------

def test_lossless_three_bus_closed_form():
    """Lossless triangle with a phase shifter: P = V1V2 sin(d)/X, Q = (V1^2 - V1V2 cos d)/X."""
    s = gridgen.PowerSystem.build(
        3,
        branches=[(0, 1, 0.0, 0.1, 0.0), (1, 2, 0.0, 0.2, 0.0), (0, 2, 0.0, 0.25, 0.0, 0.95, 0.08)],
        slack=(0, 1.0, 0.0))
    th = np.array([0.0, -0.1, -0.15])
    v = np.array([1.0, 0.98, 0.97])
    pf, qf, pt, qt = oracle.branch_flows(s, th, v)
    for k, (f, t, x, tap, sh) in enumerate([(0, 1, 0.1, 1, 0), (1, 2, 0.2, 1, 0), (0, 2, 0.25, 0.95, 0.08)]):
        e = pins.lossless_flows(v[f], v[t], th[f], th[t], x, tap, sh)
        np.testing.assert_allclose([pf[k], qf[k], pt[k], qt[k]], e, rtol=1e-13, atol=1e-14)
    fp, fq = oracle.bus_mismatch(s, th, v)
    # bus 1: P = sum over its lines of V1 Vj sin(th1 - thj)/x
    p1 = v[1] * v[0] * np.sin(th[1] - th[0]) / 0.1 + v[1] * v[2] * np.sin(th[1] - th[2]) / 0.2
    q1 = (v[1] ** 2 - v[1] * v[0] * np.cos(th[1] - th[0])) / 0.1 + \
         (v[1] ** 2 - v[1] * v[2] * np.cos(th[1] - th[2])) / 0.2
    np.testing.assert_allclose([fp[1], fq[1]], [p1, q1], rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("pl,ql,x", [(0.5, 0.2, 0.1), (1.2, 0.4, 0.05), (0.3, -0.1, 0.3)])
def test_two_bus_closed_form_solution(pl, ql, x):
    """Slack (1 /_ 0) - lossless line jx - PQ load: closed-form solution has F = 0
    and the oracle's dense Newton converges to it from flat start."""
    s = gridgen.PowerSystem.build(2, branches=[(0, 1, 0.0, x, 0.0)], loads=[(1, pl, ql)], slack=(0, 1.0, 0.0))
    v2, th2 = pins.two_bus_solution(pl, ql, x)
    xs = np.array([0.0, th2, 1.0, v2])
    F = oracle.residual(s, xs, REDUCED)
    assert np.max(np.abs(F)) < 1e-13
    # closed form of F at an arbitrary state: F_P = V2 sin(th2)/x + P_L, F_Q = (V2^2 - V2 cos th2)/x + Q_L
    xa = np.array([0.0, -0.07, 1.0, 0.96])
    Fa = oracle.residual(s, xa, REDUCED)
    np.testing.assert_allclose(Fa, [0.96 * np.sin(-0.07) / x + pl,
                                    (0.96 ** 2 - 0.96 * np.cos(-0.07)) / x + ql], rtol=1e-13)
    xn, hist = oracle.newton_dense(s, np.array([0.0, 0.0, 1.0, 1.0]))
    assert hist[-1] <= 1e-10
    np.testing.assert_allclose(xn, xs, atol=1e-10)


# --- Jacobian ------------------------------------------------------------------

@pytest.mark.parametrize("mode", [REDUCED, EXTENDED])
@pytest.mark.parametrize("k", STATES)
def test_jacobian_complex_step_small(mode, k):
    s = small_grid()
    pins.check_jacobian_complex_step(oracle, s, state(s, k, mode), mode)


@pytest.mark.parametrize("mode", [REDUCED, EXTENDED])
def test_jacobian_complex_step_three_bus(mode):
    s = three_bus()
    pins.check_jacobian_complex_step(oracle, s, state(s, 2, mode), mode)


def test_jacobian_complex_step_200():
    s = gridgen.grid_200()
    pins.check_jacobian_complex_step(oracle, s, state(s, 1), REDUCED)


@pytest.mark.parametrize("mode", [REDUCED, EXTENDED])
def test_jacobian_central_differences(mode):
    """Central differences of F against J (h = 1e-7)."""
    s = small_grid(seed=11)
    x = state(s, 5, mode)
    fm = oracle.Formulation(s, mode)
    rp, ci, jv = oracle.jacobian(s, x, mode)
    J = oracle.csr_to_dense(rp, ci, jv, fm.n_cols)
    h = 1e-7
    for c, p in enumerate(pins.column_positions(s, fm)):
        xp, xm = x.copy(), x.copy()
        xp[p] += h
        xm[p] -= h
        d = (oracle.residual(s, xp, mode) - oracle.residual(s, xm, mode)) / (2 * h)
        np.testing.assert_allclose(J[:, c], d, rtol=1e-6, atol=1e-6)


def test_formulation_dimensions():
    for s in (three_bus(), small_grid(), gridgen.grid_200()):
        pins.check_dimensions(oracle, s)


@pytest.mark.parametrize("mode", [REDUCED, EXTENDED])
def test_pattern_bruteforce(mode):
    for s in (three_bus(), small_grid(), small_grid(seed=3, n=12)):
        pins.check_pattern(oracle, s, mode)


def test_extended_rows_closed_form():
    """g_V = V - Vset, g_theta = theta_s - theta_set, with +-1 Jacobian entries (Eqs. 1-3)."""
    s = three_bus()
    x = gridgen.perturbed_state(s, 9, extended=True)
    n = 3
    fm = oracle.Formulation(s, EXTENDED)
    F = oracle.residual(s, x, EXTENDED)
    np.testing.assert_allclose(F[fm.row_gv], [x[n + 2] - 1.02, x[n + 0] - 1.01], rtol=0, atol=1e-15)
    assert abs(F[fm.row_gth] - (x[0] - 0.05)) < 1e-15
    # g_p at the slack includes -P_s; g_q at generator buses includes -Q_g
    fp, fq = oracle.bus_mismatch(s, x[:n], x[n:2 * n])
    assert abs(F[fm.row_p[0]] - (fp[0] - x[-1])) < 1e-14
    assert abs(F[fm.row_q[2]] - (fq[2] - x[2 * n])) < 1e-14
    assert abs(F[fm.row_q[0]] - (fq[0] - x[2 * n + 1])) < 1e-14
    rp, ci, jv = oracle.jacobian(s, x, EXTENDED)
    J = oracle.csr_to_dense(rp, ci, jv, fm.n_cols)
    assert J[fm.row_gv[0], fm.col_v[2]] == 1.0 and J[fm.row_gv[1], fm.col_v[0]] == 1.0
    assert J[fm.row_gth, fm.col_th[0]] == 1.0
    assert J[fm.row_q[2], fm.col_qg[0]] == -1.0 and J[fm.row_p[0], fm.col_ps] == -1.0


# --- power-flow solution and the loss invariant ---------------------------------

def test_newton_200_converges_quadratically():
    s = gridgen.grid_200()
    xs, hist = oracle.newton_dense(s, gridgen.flat_state(s))
    assert hist[-1] <= 1e-10, hist
    assert len(hist) <= 10
    # quadratic convergence over the last steps: e_{k+1} <= C e_k^2
    e = np.array(hist)
    tail = e[-3:]
    assert tail[2] <= 10 * tail[1] ** 2 + 1e-12


def test_loss_invariant_at_solution():
    """At a solution, total branch losses (Ohm's law) + shunt consumption equal
    slack generation + PV generation - load."""
    s = gridgen.grid_200()
    xs, hist = oracle.newton_dense(s, gridgen.flat_state(s))
    n = s.n_bus
    th, v = xs[:n], xs[n:2 * n]
    fp, _ = oracle.bus_mismatch(s, th, v)
    mask = np.ones(n, bool)
    mask[s.slack_bus] = False
    assert np.max(np.abs(fp[mask])) <= 1e-10
    p_slack = fp[s.slack_bus]           # the slack's generation closes its P balance
    dp, _ = pins.ohmic_losses(s, th, v)
    shunt = np.sum(s.sh_g * v[s.sh_bus] ** 2)
    lhs = dp.sum() + shunt
    rhs = p_slack + s.pv_p.sum() - s.load_p.sum()
    assert abs(lhs - rhs) <= 1e-9 * max(1.0, abs(rhs))
    assert lhs > 0


def test_extended_newton_three_bus():
    s = three_bus()
    x0 = gridgen.flat_state(s, True)
    xs, hist = oracle.newton_dense(s, x0, EXTENDED)
    assert hist[-1] <= 1e-10
    n = 3
    assert abs(xs[0] - 0.05) < 1e-12 and abs(xs[n + 0] - 1.01) < 1e-12 and abs(xs[n + 2] - 1.02) < 1e-12
    # the reduced formulation reaches the same state
    xr = np.concatenate([xs[:n], xs[n:2 * n]])
    assert np.max(np.abs(oracle.residual(s, xr, REDUCED))) < 1e-9


# --- adjoint -----------------------------------------------------------------------

@pytest.mark.parametrize("mode", [REDUCED, EXTENDED])
def test_vjp_state_complex_step(mode):
    s = small_grid(seed=5)
    x = state(s, 2, mode)
    fm = oracle.Formulation(s, mode)
    v = np.random.default_rng(1).standard_normal(fm.n_rows)
    g = oracle.vjp(s, x, v, mode)
    cs = pins.complex_step_columns(lambda xc: v @ oracle.residual(s, xc, mode), x, range(x.shape[0]))
    pins.assert_close(g["x"], cs.reshape(-1), 1e-12, 1e-11, "v^T dF/dx")


@pytest.mark.parametrize("mode", [REDUCED, EXTENDED])
def test_vjp_params_complex_step(mode):
    s = small_grid(seed=6)
    s.br_status[3] = 0
    x = state(s, 1, mode)
    fm = oracle.Formulation(s, mode)
    v = np.random.default_rng(2).standard_normal(fm.n_rows)
    g = oracle.vjp(s, x, v, mode)
    base = {"r": s.br_r, "reac": s.br_x, "b_c": s.br_b, "tap": s.br_tap}
    for out, key in (("r", "r"), ("reac", "reac"), ("b", "b_c"), ("tap", "tap")):
        cs = np.empty(s.n_branch)
        for k in range(s.n_branch):
            p = base[key].astype(complex)
            p[k] += 1e-30j
            cs[k] = (v @ oracle.residual(s, x, mode, **{key: p})).imag / 1e-30
        pins.assert_close(g[out], cs, 1e-12, 1e-11, "grad " + out)
    p0, q0 = oracle.net_injections(s)
    for out, which in (("p_inj", 0), ("q_inj", 1)):
        cs = np.empty(s.n_bus)
        for b in range(s.n_bus):
            pp, qq = p0.astype(complex), q0.astype(complex)
            (pp if which == 0 else qq)[b] += 1e-30j
            cs[b] = (v @ oracle.residual(s, x, mode, p_inj=pp, q_inj=qq)).imag / 1e-30
        pins.assert_close(g[out], cs, 1e-12, 1e-11, "grad " + out)


def test_vjp_params_central_differences_200():
    """Central differences (h = 1e-7) on a sample of branches of the 200-bus case."""
    s = gridgen.grid_200()
    x = state(s, 3)
    fm = oracle.Formulation(s, REDUCED)
    v = gridgen.gaussian_cotangents(fm.n_rows, 1)[0]
    g = oracle.vjp(s, x, v)
    h = 1e-7
    for out, key in (("r", "r"), ("reac", "reac"), ("b", "b_c"), ("tap", "tap")):
        base = {"r": s.br_r, "reac": s.br_x, "b_c": s.br_b, "tap": s.br_tap}[key]
        for k in range(0, s.n_branch, 25):
            pp, pm = base.copy(), base.copy()
            pp[k] += h
            pm[k] -= h
            d = (v @ oracle.residual(s, x, **{key: pp}) - v @ oracle.residual(s, x, **{key: pm})) / (2 * h)
            assert abs(d - g[out][k]) <= 1e-5 * max(1.0, abs(d)), (out, k, d, g[out][k])
