"""Independent checks of the CPU oracle (test helpers, no pytest here).

Each helper computes a quantity by a route that shares no formula with
``oracle/pf_oracle.py``:

* ``ybus_mismatch``: complex nodal form S = V . conj(Y V) with the textbook
  branch admittance matrix of a pi line behind an ideal phase-shifting
  transformer (the branch model the oracle writes out in polar form).
* ``ohmic_losses``: branch losses from the series current, r|I|^2 and x|I|^2.
* ``lossless_flows``: the P = V1 V2 sin(delta)/X and Q = (V1^2 - V1 V2 cos)/X
  closed forms of a lossless line / phase shifter.
* ``two_bus_solution``: the closed-form high-voltage solution of a lossless
  2-bus case (slack - line - PQ load).
* ``structural_pattern``: brute-force dense structural pattern.
* ``complex_step_columns``: derivatives of any function by the complex step.

``check_*`` functions raise AssertionError on disagreement; the mutation
test reuses them against deliberately broken copies of the oracle.
"""
from __future__ import annotations

import numpy as np

TOL_ABS = 1e-10
TOL_REL = 1e-12


def ybus_matrix(sys):
    n = sys.n_bus
    Y = np.zeros((n, n), complex)
    for k in range(sys.n_branch):
        if not sys.br_status[k]:
            continue
        f, t = int(sys.br_from[k]), int(sys.br_to[k])
        ys = 1.0 / complex(sys.br_r[k], sys.br_x[k])
        a = sys.br_tap[k] * np.exp(1j * sys.br_shift[k])
        ysh = 1j * sys.br_b[k] / 2
        Y[f, f] += (ys + ysh + sys.br_g_fr[k]) / (a * np.conj(a))
        Y[t, t] += ys + ysh + sys.br_g_to[k]
        Y[f, t] += -ys / np.conj(a)
        Y[t, f] += -ys / a
    for h in range(sys.sh_bus.shape[0]):
        b = int(sys.sh_bus[h])
        Y[b, b] += sys.sh_g[h] + 1j * sys.sh_b[h]
    return Y


def ybus_mismatch(sys, theta, V, p_inj, q_inj):
    Vc = V * np.exp(1j * theta)
    S = Vc * np.conj(ybus_matrix(sys) @ Vc)
    return S.real - p_inj, S.imag - q_inj


def injections_by_loop(sys):
    p = np.zeros(sys.n_bus)
    q = np.zeros(sys.n_bus)
    for b, pg in zip(sys.pv_bus, sys.pv_p):
        p[b] += pg
    for b, pl, ql in zip(sys.load_bus, sys.load_p, sys.load_q):
        p[b] -= pl
        q[b] -= ql
    return p, q


def ohmic_losses(sys, theta, V):
    """Per-branch (P_f + P_t, Q_f + Q_t) from the series current."""
    dp = np.zeros(sys.n_branch)
    dq = np.zeros(sys.n_branch)
    for k in range(sys.n_branch):
        if not sys.br_status[k]:
            continue
        f, t = int(sys.br_from[k]), int(sys.br_to[k])
        a = sys.br_tap[k] * np.exp(1j * sys.br_shift[k])
        vf = V[f] * np.exp(1j * theta[f]) / a          # series side of the ideal transformer
        vt = V[t] * np.exp(1j * theta[t])
        i_s = (vf - vt) / complex(sys.br_r[k], sys.br_x[k])
        i2 = abs(i_s) ** 2
        vf2 = abs(vf) ** 2
        vt2 = V[t] ** 2
        dp[k] = sys.br_r[k] * i2 + sys.br_g_fr[k] * vf2 + sys.br_g_to[k] * vt2
        dq[k] = sys.br_x[k] * i2 - sys.br_b[k] / 2 * (vf2 + vt2)
    return dp, dq


def lossless_flows(vf, vt, thf, tht, x, tap=1.0, shift=0.0):
    """Closed forms of a lossless (r = 0, b = 0) branch with tap / shift."""
    d = thf - tht - shift
    pf = vf * vt * np.sin(d) / (tap * x)
    qf = vf * vf / (tap * tap * x) - vf * vt * np.cos(d) / (tap * x)
    pt = -pf
    qt = vt * vt / x - vf * vt * np.cos(d) / (tap * x)
    return pf, qf, pt, qt


def two_bus_solution(pl, ql, x):
    """High-voltage solution (V2, theta2) of slack(1 /_ 0) --jx-- PQ load."""
    a = 1 - 2 * ql * x
    u = (a + np.sqrt(a * a - 4 * x * x * (pl * pl + ql * ql))) / 2
    v2 = np.sqrt(u)
    th2 = np.arcsin(-pl * x / v2)
    return v2, th2


def structural_pattern(sys, fm):
    """Dense boolean pattern by brute force over bus pairs."""
    n = sys.n_bus
    adj = np.eye(n, dtype=bool)
    for k in range(sys.n_branch):
        adj[sys.br_from[k], sys.br_to[k]] = True
        adj[sys.br_to[k], sys.br_from[k]] = True
    P = np.zeros((fm.n_rows, fm.n_cols), bool)
    for o in range(n):
        for j in range(n):
            if not adj[o, j]:
                continue
            for r in (fm.row_p[o], fm.row_q[o]):
                for c in (fm.col_th[j], fm.col_v[j]):
                    if r >= 0 and c >= 0:
                        P[r, c] = True
    if fm.mode == 1:
        for gi, b in enumerate(fm.gens):
            P[fm.row_q[b], fm.col_qg[gi]] = True
            P[fm.row_gv[gi], fm.col_v[b]] = True
            P[fm.row_gv[gi], fm.col_qg[gi]] = True     # g_V held at a reactive limit: Q_g - Q_lim
        P[fm.row_p[sys.slack_bus], fm.col_ps] = True
        P[fm.row_gth, fm.col_th[sys.slack_bus]] = True
    return P


def column_positions(sys, fm):
    """Position in x of each J column."""
    n = sys.n_bus
    col_x = np.full(fm.n_cols, -1, np.int64)
    for b in range(n):
        if fm.col_th[b] >= 0:
            col_x[fm.col_th[b]] = b
        if fm.col_v[b] >= 0:
            col_x[fm.col_v[b]] = n + b
    if fm.mode == 1:
        for gi in range(fm.gens.shape[0]):
            col_x[fm.col_qg[gi]] = 2 * n + gi
        col_x[fm.col_ps] = 2 * n + fm.gens.shape[0]
    return col_x


def complex_step_columns(fun, x, positions, h=1e-30):
    cols = []
    for p in positions:
        xc = np.asarray(x, complex).copy()
        xc[p] += 1j * h
        cols.append(np.asarray(fun(xc)).imag / h)
    return np.stack(cols, axis=-1)


def assert_close(a, b, rel=TOL_REL, abs_=TOL_ABS, what=""):
    a = np.asarray(a)
    b = np.asarray(b)
    err = np.abs(a - b)
    bound = abs_ + rel * np.abs(b)
    bad = err > bound
    if bad.any():
        i = np.unravel_index(np.argmax(err - bound), err.shape)
        raise AssertionError(f"{what}: {int(bad.sum())} entries off; worst at {i}: {a[i]!r} vs {b[i]!r}")


# ---------------------------------------------------------------------------
# checks usable against any oracle module (the real one or a mutated copy)
# ---------------------------------------------------------------------------

def check_ybus(orc, sys, x):
    n = sys.n_bus
    theta, V = x[:n], x[n:2 * n]
    p, q = injections_by_loop(sys)
    fp, fq = orc.bus_mismatch(sys, theta, V)
    yp, yq = ybus_mismatch(sys, theta, V, p, q)
    assert_close(fp, yp, 1e-12, 1e-11, "P mismatch vs Y-bus")
    assert_close(fq, yq, 1e-12, 1e-11, "Q mismatch vs Y-bus")


def check_ohmic(orc, sys, x):
    n = sys.n_bus
    theta, V = x[:n], x[n:2 * n]
    pf, qf, pt, qt = orc.branch_flows(sys, theta, V)
    dp, dq = ohmic_losses(sys, theta, V)
    assert_close(pf + pt, dp, 1e-12, 1e-11, "P losses vs r|I|^2")
    assert_close(qf + qt, dq, 1e-12, 1e-11, "Q losses vs x|I|^2")


def check_jacobian_complex_step(orc, sys, x, mode):
    fm = orc.Formulation(sys, mode)
    rp, ci, jv = orc.jacobian(sys, x, mode)
    J = orc.csr_to_dense(rp, ci, jv, fm.n_cols)
    col_x = column_positions(sys, fm)
    Jc = complex_step_columns(lambda xc: orc.residual(sys, xc, mode), x, col_x)
    assert_close(J, Jc, 1e-12, 1e-11, "J vs complex step")
    return J, Jc


def check_pattern(orc, sys, mode):
    fm = orc.Formulation(sys, mode)
    n = sys.n_bus
    x = np.concatenate([np.zeros(n), np.ones(n)])
    if mode == 1:
        x = np.concatenate([x, np.zeros(sys.n_pv + 2)])
    rp, ci, _ = orc.jacobian(sys, x, mode)
    P = np.zeros((fm.n_rows, fm.n_cols), bool)
    for i in range(fm.n_rows):
        cols = ci[rp[i]:rp[i + 1]]
        assert np.all(np.diff(cols) > 0), "columns not strictly ascending"
        P[i, cols] = True
    Pb = structural_pattern(sys, fm)
    if not np.array_equal(P, Pb):
        raise AssertionError(f"pattern differs in {(P != Pb).sum()} places")


def check_dimensions(orc, sys):
    """Reduced J is (2N - N_PV - 2)^2 (P rows of the N-1 non-slack buses, Q rows
    of the N - N_PV - 1 PQ buses); extended J is (2N + N_gen + 1)^2 with
    N_gen = N_PV + 1 (Eqs. 1-3).  P rows follow ascending bus order."""
    n, npv = sys.n_bus, len(set(int(b) for b in sys.pv_bus) - {sys.slack_bus})
    fr = orc.Formulation(sys, 0)
    if (fr.n_rows, fr.n_cols) != (2 * n - npv - 2, 2 * n - npv - 2):
        raise AssertionError(f"reduced size {fr.n_rows} != {2 * n - npv - 2}")
    pq = [b for b in range(n) if b != sys.slack_bus and b not in set(int(v) for v in sys.pv_bus)]
    if list(fr.row_q[pq]) != list(range(n - 1, n - 1 + len(pq))) or np.any(np.delete(fr.row_q, pq) >= 0):
        raise AssertionError("reduced Q rows are not the PQ buses in ascending order")
    ns = [b for b in range(n) if b != sys.slack_bus]
    if list(fr.row_p[ns]) != list(range(n - 1)) or fr.row_p[sys.slack_bus] != -1:
        raise AssertionError("reduced P rows are not the non-slack buses in ascending order")
    fe = orc.Formulation(sys, 1)
    if fe.n_rows != 2 * n + sys.n_pv + 2:
        raise AssertionError("extended size")
