"""Plain FP64 CPU oracle for power-flow residual / Jacobian evaluation.

TEST INFRASTRUCTURE ONLY.  This module is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the CPU-baseline / reference arm of
``bench.py``; the library path never calls it and shares no code with it.

It is the plain definition of what tasks (1) and (2) of Newton power flow
compute (Sec. I): the bus power mismatches g(y) and the nonzero entries of
their Jacobian, written as a loop over models (Sec. II-A: Bus, PQ load, PV
generator, Slack, Line / transformer, Shunt) in polar coordinates.  Loops
over branches are numpy vector operations over the branch arrays; per-bus
sums are ``np.add.at`` scatters in branch order.  Nothing is blocked, fused
or reordered beyond that.  Every function is written to accept complex
inputs as well (no abs / conj / comparisons on the values), so the tests
can differentiate it by the complex-step method.

Readings of the paper used here (the paper prints only the active-power line
of the branch model, Eq. 4):
  * Branch model: series admittance g + jb = 1 / (r + jx); charging b_c split
    b_c/2 per end; end conductances g_fr, g_to (g_{L,h}, g_{L,k} of Eq. 4);
    off-nominal tap tau and phase shift phi on the from side;
    delta = theta_f - theta_t - phi.  With tau = 1, phi = 0 and b_c = 0 the P
    lines are exactly Eq. (4).
  * Residual sign: F = power flowing out into branches + shunt consumption
    + load - generation (the sign of Eq. 4, which counts P_h as leaving h).
  * Extended formulation (Eqs. 1-3): rows [g_p(N), g_q(N), g_V(gens), g_theta],
    columns [theta(N), V(N), Q_g(gens), P_s]; generators are the PV units in
    input order followed by the slack; g_V = V - Vset, g_theta = theta_s - theta_set.
  * Reactive limits in the extended formulation (Sec. II-A: the same
    formulation serves before and after a PV generator switches to a PQ
    load): a generator in voltage control has g_V = V - Vset; one held at a
    reactive limit has g_V = Q_g - Q_lim instead.  Its g_V row always carries
    both entries, dg_V/dV and dg_V/dQ_g (one of them an explicit zero), so
    switching never changes the pattern.
  * Reduced (classic) formulation: rows/columns [P/theta of non-slack buses,
    Q/V of PQ-type buses], each in ascending bus order.
  * Jacobian pattern: the structural union of all model contributions; the
    four diagonal entries of a bus are present whenever their row and column
    exist; out-of-service branches keep their entries (value 0).
"""
from __future__ import annotations

import numpy as np

REDUCED = 0
EXTENDED = 1


# ---------------------------------------------------------------------------
# branch model (Sec. II-A; Sec. II-B, Eq. 4)
# ---------------------------------------------------------------------------

def series_admittance(r, x):
    """g + jb = 1/(r + jx): g = r/(r^2+x^2), b = -x/(r^2+x^2)."""
    d = r * r + x * x
    return r / d, -x / d


def branch_flows(sys, theta, V, r=None, reac=None, b_c=None, tap=None, status=None):
    """Terminal powers of every branch, counted as leaving the terminal bus.

    P_f, Q_f at the from bus and P_t, Q_t at the to bus (Eq. 4 plus the
    reactive lines, tap and phase shift of the pi / transformer model).
    Parameter arrays (``reac`` is the series reactance) default to the system's.
    """
    r = sys.br_r if r is None else r
    x = sys.br_x if reac is None else reac
    b_c = sys.br_b if b_c is None else b_c
    tau = sys.br_tap if tap is None else tap
    on = sys.br_status if status is None else status
    f, t = sys.br_from, sys.br_to
    g, b = series_admittance(r, x)
    delta = theta[f] - theta[t] - sys.br_shift
    cd, sd = np.cos(delta), np.sin(delta)
    vf, vt = V[f], V[t]
    vv = vf * vt / tau
    pf = vf * vf * (g + sys.br_g_fr) / (tau * tau) - vv * (g * cd + b * sd)
    qf = -vf * vf * (b + b_c / 2) / (tau * tau) - vv * (g * sd - b * cd)
    pt = vt * vt * (g + sys.br_g_to) - vv * (g * cd - b * sd)
    qt = -vt * vt * (b + b_c / 2) + vv * (g * sd + b * cd)
    return pf * on, qf * on, pt * on, qt * on


def branch_partials(sys, theta, V):
    """The 16 partial derivatives of (P_f, Q_f, P_t, Q_t) with respect to
    (theta_f, theta_t, V_f, V_t), differentiated by hand from ``branch_flows``.

    Returns a dict keyed like 'Pf_thf', 'Qt_Vf', ...
    """
    f, t = sys.br_from, sys.br_to
    g, b = series_admittance(sys.br_r, sys.br_x)
    tau, on = sys.br_tap, sys.br_status
    bc2 = sys.br_b / 2
    delta = theta[f] - theta[t] - sys.br_shift
    cd, sd = np.cos(delta), np.sin(delta)
    vf, vt = V[f], V[t]
    vv = vf * vt / tau
    d = {}
    # P_f = vf^2 (g+g_fr)/tau^2 - (vf vt/tau)(g cos + b sin)
    d["Pf_thf"] = vv * (g * sd - b * cd)
    d["Pf_tht"] = -vv * (g * sd - b * cd)
    d["Pf_Vf"] = 2 * vf * (g + sys.br_g_fr) / (tau * tau) - (vt / tau) * (g * cd + b * sd)
    d["Pf_Vt"] = -(vf / tau) * (g * cd + b * sd)
    # Q_f = -vf^2 (b + bc/2)/tau^2 - (vf vt/tau)(g sin - b cos)
    d["Qf_thf"] = -vv * (g * cd + b * sd)
    d["Qf_tht"] = vv * (g * cd + b * sd)
    d["Qf_Vf"] = -2 * vf * (b + bc2) / (tau * tau) - (vt / tau) * (g * sd - b * cd)
    d["Qf_Vt"] = -(vf / tau) * (g * sd - b * cd)
    # P_t = vt^2 (g+g_to) - (vf vt/tau)(g cos - b sin)
    d["Pt_thf"] = vv * (g * sd + b * cd)
    d["Pt_tht"] = -vv * (g * sd + b * cd)
    d["Pt_Vf"] = -(vt / tau) * (g * cd - b * sd)
    d["Pt_Vt"] = 2 * vt * (g + sys.br_g_to) - (vf / tau) * (g * cd - b * sd)
    # Q_t = -vt^2 (b + bc/2) + (vf vt/tau)(g sin + b cos)
    d["Qt_thf"] = vv * (g * cd - b * sd)
    d["Qt_tht"] = -vv * (g * cd - b * sd)
    d["Qt_Vf"] = (vt / tau) * (g * sd + b * cd)
    d["Qt_Vt"] = -2 * vt * (b + bc2) + (vf / tau) * (g * sd + b * cd)
    return {k: v * on for k, v in d.items()}


def branch_param_partials(sys, theta, V):
    """Partials of (P_f, Q_f, P_t, Q_t) with respect to (r, x, b_c, tap) of
    the same branch: chain rule through g = r/D, b = -x/D, D = r^2 + x^2.

    Returns a dict keyed like 'Pf_r', 'Qt_tap', ...
    """
    f, t = sys.br_from, sys.br_to
    r, x = sys.br_r, sys.br_x
    dd = r * r + x * x
    g, b = r / dd, -x / dd
    dg_dr, dg_dx = (x * x - r * r) / (dd * dd), -2 * r * x / (dd * dd)
    db_dr, db_dx = 2 * r * x / (dd * dd), (x * x - r * r) / (dd * dd)
    tau, on = sys.br_tap, sys.br_status
    bc2 = sys.br_b / 2
    delta = theta[f] - theta[t] - sys.br_shift
    cd, sd = np.cos(delta), np.sin(delta)
    vf, vt = V[f], V[t]
    vv = vf * vt / tau
    # derivatives with respect to the series g and b
    Pf_g, Pf_b = vf * vf / (tau * tau) - vv * cd, -vv * sd
    Qf_g, Qf_b = -vv * sd, -vf * vf / (tau * tau) + vv * cd
    Pt_g, Pt_b = vt * vt - vv * cd, vv * sd
    Qt_g, Qt_b = vv * sd, -vt * vt + vv * cd
    out = {}
    for name, dg, db in (("r", dg_dr, db_dr), ("x", dg_dx, db_dx)):
        out["Pf_" + name] = Pf_g * dg + Pf_b * db
        out["Qf_" + name] = Qf_g * dg + Qf_b * db
        out["Pt_" + name] = Pt_g * dg + Pt_b * db
        out["Qt_" + name] = Qt_g * dg + Qt_b * db
    zero = 0 * vf
    out["Pf_bc"], out["Qf_bc"] = zero, -vf * vf / (2 * tau * tau)
    out["Pt_bc"], out["Qt_bc"] = zero, -vt * vt / 2
    vv2 = vf * vt / (tau * tau)
    out["Pf_tap"] = -2 * vf * vf * (g + sys.br_g_fr) / tau ** 3 + vv2 * (g * cd + b * sd)
    out["Qf_tap"] = 2 * vf * vf * (b + bc2) / tau ** 3 + vv2 * (g * sd - b * cd)
    out["Pt_tap"] = vv2 * (g * cd - b * sd)
    out["Qt_tap"] = -vv2 * (g * sd + b * cd)
    return {k: v * on for k, v in out.items()}


# ---------------------------------------------------------------------------
# bus models and the per-bus join (Sec. II-A: each branch's terminal injections
# are evaluated branch by branch, then added into the two buses it joins)
# ---------------------------------------------------------------------------

def net_injections(sys):
    """Per-bus P_inj = sum(P_g of PV units) - sum(P_load), Q_inj = -sum(Q_load)."""
    n = sys.n_bus
    p = np.zeros(n)
    q = np.zeros(n)
    np.add.at(p, sys.pv_bus, sys.pv_p)
    np.add.at(p, sys.load_bus, -sys.load_p)
    np.add.at(q, sys.load_bus, -sys.load_q)
    return p, q


def bus_mismatch(sys, theta, V, p_inj=None, q_inj=None, **branch_params):
    """Full active / reactive mismatch of every bus (no formulation applied):
    F_P = sum of outgoing P + g_sh V^2 - P_inj, F_Q = sum of outgoing Q - b_sh V^2 - Q_inj."""
    n = sys.n_bus
    dt = np.result_type(theta, V, *(v for v in branch_params.values() if v is not None),
                        *(v for v in (p_inj, q_inj) if v is not None))
    pf, qf, pt, qt = branch_flows(sys, theta, V, **branch_params)
    fp = np.zeros(n, dtype=dt)
    fq = np.zeros(n, dtype=dt)
    np.add.at(fp, sys.br_from, pf)
    np.add.at(fp, sys.br_to, pt)
    np.add.at(fq, sys.br_from, qf)
    np.add.at(fq, sys.br_to, qt)
    vs = V[sys.sh_bus]
    np.add.at(fp, sys.sh_bus, sys.sh_g * vs * vs)
    np.add.at(fq, sys.sh_bus, -sys.sh_b * vs * vs)
    if p_inj is None or q_inj is None:
        p0, q0 = net_injections(sys)
        p_inj = p0 if p_inj is None else p_inj
        q_inj = q0 if q_inj is None else q_inj
    return fp - p_inj, fq - q_inj


# ---------------------------------------------------------------------------
# formulations (Sec. II-A, Eqs. 1-3, and the classic reduced form)
# ---------------------------------------------------------------------------

class Formulation:
    """Row / column index maps.  ``-1`` marks a row or column that does not exist.

    row_p[b], row_q[b]  : F row of the bus's active / reactive mismatch
    col_th[b], col_v[b] : J column of the bus's angle / magnitude
    gens                : generator buses (PV units in input order, then slack),
                          extended formulation only
    """

    def __init__(self, sys, mode):
        n = sys.n_bus
        s = sys.slack_bus
        self.mode = mode
        self.n_bus = n
        is_pv = np.zeros(n, bool)
        is_pv[sys.pv_bus] = True
        is_pv[s] = False
        self.bus_type = np.zeros(n, np.int8)      # 0 PQ, 1 PV, 2 slack
        self.bus_type[is_pv] = 1
        self.bus_type[s] = 2
        if mode == REDUCED:
            non_slack = [b for b in range(n) if b != s]
            pq = [b for b in range(n) if self.bus_type[b] == 0]
            self.row_p = np.full(n, -1, np.int64)
            self.row_q = np.full(n, -1, np.int64)
            self.row_p[non_slack] = np.arange(len(non_slack))
            self.row_q[pq] = len(non_slack) + np.arange(len(pq))
            self.n_rows = len(non_slack) + len(pq)
            self.gens = np.zeros(0, np.int64)
            self.row_gv = np.zeros(0, np.int64)
            self.row_gth = -1
            self.col_qg = np.zeros(0, np.int64)
            self.col_ps = -1
        elif mode == EXTENDED:
            self.row_p = np.arange(n, dtype=np.int64)
            self.row_q = n + np.arange(n, dtype=np.int64)
            self.gens = np.concatenate([np.asarray(sys.pv_bus, np.int64), [s]])
            ng = self.gens.shape[0]
            self.row_gv = 2 * n + np.arange(ng)
            self.row_gth = 2 * n + ng
            self.col_qg = 2 * n + np.arange(ng)
            self.col_ps = 2 * n + ng
            self.n_rows = 2 * n + ng + 1
        else:
            raise ValueError("mode must be REDUCED or EXTENDED")
        self.col_th = self.row_p.copy()
        self.col_v = self.row_q.copy()
        self.n_cols = self.n_rows

    def state_index(self):
        """Position in the state vector x of theta_b (b) and V_b (N + b)."""
        n = self.n_bus
        return np.arange(n), n + np.arange(n)


def split_state(sys, x, mode):
    n = sys.n_bus
    theta, V = x[:n], x[n:2 * n]
    if mode == EXTENDED:
        ng = sys.n_pv + 1
        return theta, V, x[2 * n:2 * n + ng], x[2 * n + ng]
    return theta, V, None, None


def residual(sys, x, mode=REDUCED, p_inj=None, q_inj=None, gen_mode=None, gen_qlim=None, **branch_params):
    """Task (1): the residual vector F in the formulation's row order.

    ``x`` is the full state [theta(N), V(N)] (+ [Q_g, P_s] extended); in the
    reduced formulation the slack angle and the PV / slack magnitudes are read
    from x as fixed values.  Extended formulation: ``gen_mode[i]`` != 0 holds
    generator i at the reactive output ``gen_qlim[i]`` (g_V = Q_g - Q_lim).
    """
    fm = Formulation(sys, mode)
    theta, V, qg, ps = split_state(sys, x, mode)
    fp, fq = bus_mismatch(sys, theta, V, p_inj, q_inj, **branch_params)
    dt = np.result_type(fp, x)
    out = np.zeros(fm.n_rows, dtype=dt)
    if mode == EXTENDED:
        fp = fp.copy()
        fq = fq.copy()
        fp[sys.slack_bus] -= ps
        np.add.at(fq, fm.gens, -qg)
        vset = np.concatenate([sys.pv_vset, [sys.slack_vset]])
        out[fm.row_gv] = V[fm.gens] - vset
        if gen_mode is not None:
            held = np.asarray(gen_mode) != 0
            out[fm.row_gv[held]] = qg[held] - np.asarray(gen_qlim)[held]
        out[fm.row_gth] = theta[sys.slack_bus] - sys.slack_theta
    hp = fm.row_p >= 0
    hq = fm.row_q >= 0
    out[fm.row_p[hp]] = fp[hp]
    out[fm.row_q[hq]] = fq[hq]
    return out


# ---------------------------------------------------------------------------
# Jacobian (task 2)
# ---------------------------------------------------------------------------

def _triplets(sys, x, mode, state_columns, gen_mode=None):
    """All (row, col, value) contributions of every model.

    ``state_columns``: columns are positions in x (theta_b -> b, V_b -> N+b,
    extended extras -> their x positions) instead of formulation unknowns.
    """
    fm = Formulation(sys, mode)
    n = sys.n_bus
    theta, V, _, _ = split_state(sys, x, mode)
    d = branch_partials(sys, theta, V)
    f, t = np.asarray(sys.br_from, np.int64), np.asarray(sys.br_to, np.int64)
    if state_columns:
        cth = np.arange(n)
        cv = n + np.arange(n)
        if mode == EXTENDED:
            cqg, cps = fm.col_qg, fm.col_ps
        else:
            cqg, cps = None, None
    else:
        cth, cv = fm.col_th, fm.col_v
        cqg, cps = fm.col_qg, fm.col_ps
    rows, cols, vals = [], [], []

    def put(r, c, v):
        r = np.asarray(r)
        c = np.asarray(c)
        v = np.broadcast_to(v, r.shape)
        ok = (r >= 0) & (c >= 0)
        rows.append(r[ok])
        cols.append(c[ok])
        vals.append(v[ok])

    for end, own in (("f", f), ("t", t)):
        P, Q = "P" + end, "Q" + end
        for var, bus, cmap in (("thf", f, cth), ("tht", t, cth), ("Vf", f, cv), ("Vt", t, cv)):
            put(fm.row_p[own], cmap[bus], d[P + "_" + var])
            put(fm.row_q[own], cmap[bus], d[Q + "_" + var])
    # shunts: d(g V^2)/dV = 2 g V ; d(-b V^2)/dV = -2 b V
    sb = np.asarray(sys.sh_bus, np.int64)
    put(fm.row_p[sb], cv[sb], 2 * sys.sh_g * V[sb])
    put(fm.row_q[sb], cv[sb], -2 * sys.sh_b * V[sb])
    # the four diagonal entries always exist when row and column do
    allb = np.arange(n)
    zero = np.zeros(n, dtype=np.result_type(V))
    for rmap in (fm.row_p, fm.row_q):
        for cmap in (cth, cv):
            put(rmap[allb], cmap[allb], zero)
    if mode == EXTENDED:
        ng = fm.gens.shape[0]
        one = np.ones(ng)
        put(fm.row_q[fm.gens], cqg, -one)                   # g_q gets -Q_g
        put([fm.row_p[sys.slack_bus]], [cps], [-1.0])        # g_p at slack gets -P_s
        held = np.zeros(ng, bool) if gen_mode is None else np.asarray(gen_mode) != 0
        put(fm.row_gv, cv[fm.gens], np.where(held, 0.0, 1.0))   # g_V = V - Vset
        put(fm.row_gv, cqg, np.where(held, 1.0, 0.0))           # g_V = Q_g - Q_lim when held
        put([fm.row_gth], [cth[sys.slack_bus]], [1.0])       # g_theta = theta_s - theta_set
    return (np.concatenate(rows), np.concatenate(cols),
            np.concatenate([np.asarray(v) for v in vals]))


def _coo_to_csr(rows, cols, vals, n_rows, n_cols):
    """Sum duplicate (row, col) pairs; keep explicit zeros; ascending columns."""
    key = rows.astype(np.int64) * n_cols + cols.astype(np.int64)
    uk, inv = np.unique(key, return_inverse=True)
    data = np.zeros(uk.shape[0], dtype=vals.dtype)
    np.add.at(data, inv, vals)
    r = uk // n_cols
    colind = (uk % n_cols).astype(np.int32)
    rowptr = np.zeros(n_rows + 1, np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr).astype(np.int32)
    return rowptr, colind, data


def jacobian(sys, x, mode=REDUCED, gen_mode=None):
    """Task (2): CSR (rowptr, colind, values) of dF/d(unknowns), ascending columns."""
    fm = Formulation(sys, mode)
    r, c, v = _triplets(sys, x, mode, state_columns=False, gen_mode=gen_mode)
    return _coo_to_csr(r, c, v, fm.n_rows, fm.n_cols)


def jacobian_state(sys, x, mode=REDUCED, gen_mode=None):
    """CSR of dF/dx over every entry of the state vector x (all theta, all V,
    and the extended extras), used for vector-Jacobian products."""
    fm = Formulation(sys, mode)
    r, c, v = _triplets(sys, x, mode, state_columns=True, gen_mode=gen_mode)
    n_x = x.shape[0]
    return _coo_to_csr(r, c, v, fm.n_rows, n_x)


def csr_to_dense(rowptr, colind, vals, n_cols):
    n_rows = rowptr.shape[0] - 1
    out = np.zeros((n_rows, n_cols), dtype=vals.dtype)
    for i in range(n_rows):
        out[i, colind[rowptr[i]:rowptr[i + 1]]] += vals[rowptr[i]:rowptr[i + 1]]
    return out


def csr_matvec_t(rowptr, colind, vals, v, n_cols):
    """J^T v for a CSR J."""
    out = np.zeros(n_cols, dtype=np.result_type(vals, v))
    rows = np.repeat(np.arange(rowptr.shape[0] - 1), np.diff(rowptr))
    np.add.at(out, colind, vals * v[rows])
    return out


# ---------------------------------------------------------------------------
# vector-Jacobian products (adjoint)
# ---------------------------------------------------------------------------

def vjp(sys, x, v, mode=REDUCED, gen_mode=None):
    """v^T dF/d(x, P_inj, Q_inj, r, x_branch, b_c, tap).

    Returns dict with 'x' (len(x)), 'p_inj', 'q_inj' (N) and 'r', 'reac',
    'b', 'tap' (M).  dF_P/dP_inj = -1 and dF_Q/dQ_inj = -1 on existing rows.
    """
    fm = Formulation(sys, mode)
    n = sys.n_bus
    rp, ci, jv = jacobian_state(sys, x, mode, gen_mode)
    out = {"x": csr_matvec_t(rp, ci, jv, v, x.shape[0])}
    vp = np.zeros(n)
    vq = np.zeros(n)
    hp, hq = fm.row_p >= 0, fm.row_q >= 0
    vp[hp] = v[fm.row_p[hp]]
    vq[hq] = v[fm.row_q[hq]]
    out["p_inj"] = -vp
    out["q_inj"] = -vq
    theta, V, _, _ = split_state(sys, x, mode)
    d = branch_param_partials(sys, theta, V)
    f, t = sys.br_from, sys.br_to
    for name, key in (("r", "r"), ("reac", "x"), ("b", "bc"), ("tap", "tap")):
        out[name] = (vp[f] * d["Pf_" + key] + vq[f] * d["Qf_" + key]
                     + vp[t] * d["Pt_" + key] + vq[t] * d["Qt_" + key])
    return out


# ---------------------------------------------------------------------------
# canonical index maps (the integer maps a pattern builder must reproduce)
# ---------------------------------------------------------------------------

def incidence_lists(sys):
    """Per-bus incidence list: every branch end at bus o, ordered by
    (other bus, branch id).  Entry code = 2*branch + end (end 0 = from, 1 = to).
    Returns (ptr[N+1], code[2M], other[2M])."""
    n, m = sys.n_bus, sys.n_branch
    f = np.asarray(sys.br_from, np.int64)
    t = np.asarray(sys.br_to, np.int64)
    own = np.concatenate([f, t])
    other = np.concatenate([t, f])
    code = np.concatenate([2 * np.arange(m), 2 * np.arange(m) + 1])
    order = np.lexsort((code // 2, other, own))   # last key is primary
    ptr = np.zeros(n + 1, np.int64)
    np.add.at(ptr, own + 1, 1)
    ptr = np.cumsum(ptr)
    return ptr.astype(np.int32), code[order].astype(np.int32), other[order].astype(np.int32)


def contribution_lists(sys, mode=REDUCED):
    """Per-nonzero contribution list of J, in the order of ``jacobian``'s CSR.

    Sources of the nonzero (row of bus o, column of bus j):
      * branch-end partials: incidence-list positions e of bus o whose other
        end is j (j != o), or all incidences of o (j == o), in list order;
      * shunts (only in the V-diagonal entries): 2M + shunt index, ascending;
      * -1 for a constant +-1 entry of the extended formulation.
    Returns (ptr[nnz+1], src[...]).
    """
    fm = Formulation(sys, mode)
    n = sys.n_bus
    x0 = np.concatenate([np.zeros(n), np.ones(n)])
    if mode == EXTENDED:
        x0 = np.concatenate([x0, np.zeros(sys.n_pv + 2)])
    rowptr, colind, _ = jacobian(sys, x0, mode)
    iptr, _, other = incidence_lists(sys)
    n_inc = other.shape[0]
    # inverse maps row -> (bus, kind), col -> (bus, kind)
    row_bus = np.full(fm.n_rows, -1)
    row_kind = np.full(fm.n_rows, -1)   # 0 P, 1 Q, 2 gV, 3 gtheta
    for kind, rmap in ((0, fm.row_p), (1, fm.row_q)):
        ok = rmap >= 0
        row_bus[rmap[ok]] = np.arange(n)[ok]
        row_kind[rmap[ok]] = kind
    col_bus = np.full(fm.n_cols, -1)
    col_kind = np.full(fm.n_cols, -1)   # 0 theta, 1 V, 2 Qg, 3 Ps
    for kind, cmap in ((0, fm.col_th), (1, fm.col_v)):
        ok = cmap >= 0
        col_bus[cmap[ok]] = np.arange(n)[ok]
        col_kind[cmap[ok]] = kind
    if mode == EXTENDED:
        row_kind[fm.row_gv] = 2
        row_kind[fm.row_gth] = 3
        col_kind[fm.col_qg] = 2
        col_kind[fm.col_ps] = 3
    sh_of_bus = [[] for _ in range(n)]
    for h, b in enumerate(sys.sh_bus):
        sh_of_bus[int(b)].append(2 * sys.n_branch + h)
    ptr = [0]
    src = []
    for i in range(fm.n_rows):
        for k in range(rowptr[i], rowptr[i + 1]):
            j = colind[k]
            rk, ck = row_kind[i], col_kind[j]
            if rk >= 2 or ck >= 2:
                src.append(-1)
            else:
                o, jb = row_bus[i], col_bus[j]
                lo, hi = iptr[o], iptr[o + 1]
                if jb == o:
                    src.extend(range(lo, hi))
                    if ck == 1:
                        src.extend(sh_of_bus[o])
                else:
                    src.extend(e for e in range(lo, hi) if other[e] == jb)
            ptr.append(len(src))
    assert n_inc == 2 * sys.n_branch
    return np.asarray(ptr, np.int64), np.asarray(src, np.int32)


# ---------------------------------------------------------------------------
# dense Newton (tiny grids only; task (3) by a library dense solve)
# ---------------------------------------------------------------------------

def newton_dense(sys, x0, mode=REDUCED, tol=1e-10, max_iter=30, gen_mode=None, gen_qlim=None):
    """Newton iterations on the formulation's unknowns with a dense solve.

    Returns (x, history of ||F||_inf).  Stops when ||F||_inf <= tol.
    """
    fm = Formulation(sys, mode)
    n = sys.n_bus
    x = np.array(x0, dtype=float)
    # position in x of every J column
    col_x = np.full(fm.n_cols, -1, np.int64)
    ok = fm.col_th >= 0
    col_x[fm.col_th[ok]] = np.arange(n)[ok]
    ok = fm.col_v >= 0
    col_x[fm.col_v[ok]] = n + np.arange(n)[ok]
    if mode == EXTENDED:
        col_x[fm.col_qg] = 2 * n + np.arange(fm.gens.shape[0])
        col_x[fm.col_ps] = 2 * n + fm.gens.shape[0]
    hist = []
    for _ in range(max_iter):
        F = residual(sys, x, mode, gen_mode=gen_mode, gen_qlim=gen_qlim)
        hist.append(float(np.max(np.abs(F))) if F.size else 0.0)
        if hist[-1] <= tol:
            break
        rp, ci, jv = jacobian(sys, x, mode, gen_mode)
        J = csr_to_dense(rp, ci, jv, fm.n_cols)
        x[col_x] -= np.linalg.solve(J, F)
    return x, hist


def newton_qlim(sys, x0, q_min, q_max, tol=1e-10, max_iter=30, max_switch_rounds=20):
    """Extended-formulation Newton with reactive limits (Sec. II-A: limits are
    checked between solves and a generator that violates one is held at it,
    the formulation unchanged).  Generators in voltage control whose Q_g ends
    above q_max or below q_min are switched to that limit and the system is
    solved again, until no generator in voltage control violates a limit.
    Generators are the PV units in input order, then the slack.

    Returns (x, gen_mode, gen_qlim, rounds): gen_mode 0 = voltage control,
    1 = held at q_max, 2 = held at q_min.
    """
    n = sys.n_bus
    ng = sys.n_pv + 1
    q_min = np.asarray(q_min, float)
    q_max = np.asarray(q_max, float)
    gen_mode = np.zeros(ng, np.int8)
    gen_qlim = np.zeros(ng)
    x = np.array(x0, dtype=float)
    for rounds in range(1, max_switch_rounds + 1):
        x, hist = newton_dense(sys, x, EXTENDED, tol, max_iter, gen_mode, gen_qlim)
        if hist[-1] > tol:
            raise RuntimeError("Newton did not converge")
        qg = x[2 * n:2 * n + ng]
        hi = (gen_mode == 0) & (qg > q_max)
        lo = (gen_mode == 0) & (qg < q_min)
        if not (hi.any() or lo.any()):
            return x, gen_mode, gen_qlim, rounds
        gen_mode[hi] = 1
        gen_qlim[hi] = q_max[hi]
        gen_mode[lo] = 2
        gen_qlim[lo] = q_min[lo]
    raise RuntimeError("reactive-limit switching did not settle")


# ---------------------------------------------------------------------------
# fast decoupled iterations (Sec. V names the Fast Decoupled method as future
# work; the XB variant of Stott and Alsac, with van Amerongen's choice of
# which matrix drops the resistances)
# ---------------------------------------------------------------------------

def fdlf_matrices(sys):
    """(B', B'') of the XB fast decoupled method, dense, reduced-formulation order.

    B' (rows / columns: non-slack buses): built from 1/x of every in-service
    branch only (resistance, charging, taps, shifts and shunts ignored);
    B'' (rows / columns: PQ-type buses): -Im(Y_bus) with phase shifts set to
    zero (series admittance, charging, taps and shunts kept).
    """
    fm = Formulation(sys, REDUCED)
    n = sys.n_bus
    on = np.asarray(sys.br_status) != 0
    f = np.asarray(sys.br_from, np.int64)[on]
    t = np.asarray(sys.br_to, np.int64)[on]
    x = np.asarray(sys.br_x, float)[on]
    r = np.asarray(sys.br_r, float)[on]
    bc = np.asarray(sys.br_b, float)[on]
    tau = np.asarray(sys.br_tap, float)[on]
    B1 = np.zeros((n, n))
    y1 = 1.0 / x
    np.add.at(B1, (f, f), y1)
    np.add.at(B1, (t, t), y1)
    np.add.at(B1, (f, t), -y1)
    np.add.at(B1, (t, f), -y1)
    bs = -x / (r * r + x * x)                          # Im of the series admittance 1 / (r + jx)
    B2 = np.zeros((n, n))
    np.add.at(B2, (f, f), -(bs + bc / 2) / (tau * tau))
    np.add.at(B2, (t, t), -(bs + bc / 2))
    np.add.at(B2, (f, t), bs / tau)
    np.add.at(B2, (t, f), bs / tau)
    np.add.at(B2, (np.asarray(sys.sh_bus, np.int64), np.asarray(sys.sh_bus, np.int64)), -np.asarray(sys.sh_b))
    ns = np.argsort(np.where(fm.row_p >= 0, fm.row_p, n + 1))[: int(np.sum(fm.row_p >= 0))]
    pq = np.argsort(np.where(fm.row_q >= 0, fm.row_q, 2 * n + 1))[: int(np.sum(fm.row_q >= 0))]
    return B1[np.ix_(ns, ns)], B2[np.ix_(pq, pq)], ns, pq


def fdlf(sys, x0, tol=1e-10, max_iter=100):
    """Fast decoupled iterations (reduced formulation): with the mismatches
    F = P_out - P_spec (this module's sign), each iteration solves
    B' dtheta = -F_P / V and updates theta, re-evaluates F, solves
    B'' dV = -F_Q / V and updates V.  Returns (x, history of ||F||_inf), the
    norm taken before each iteration; stops at ||F||_inf <= tol.
    """
    n = sys.n_bus
    fm = Formulation(sys, REDUCED)
    B1, B2, ns, pq = fdlf_matrices(sys)
    x = np.array(x0, dtype=float)
    hist = []
    for _ in range(max_iter):
        F = residual(sys, x)
        hist.append(float(np.max(np.abs(F))) if F.size else 0.0)
        if hist[-1] <= tol:
            break
        x[ns] += np.linalg.solve(B1, -F[fm.row_p[ns]] / x[n + ns])
        F = residual(sys, x)
        x[n + pq] += np.linalg.solve(B2, -F[fm.row_q[pq]] / x[n + pq])
    return x, hist

