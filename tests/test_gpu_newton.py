"""Newton iterations around the hot path (pf_newton: this library's F, J,
convergence test and update kernels; cuSOLVER's sparse QR for the solve)
against the oracle's dense Newton and the 2-bus closed form.  GPU only."""
import math

import numpy as np
import pytest
import torch

import gridgen
import oracle
from oracle import EXTENDED, REDUCED
from tests.gpu_common import assert_tol, two_bus, with_outage

pytestmark = pytest.mark.gpu
MNAME = {REDUCED: "reduced", EXTENDED: "extended"}


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2011_11880_gb300 as p
    return p


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("solver", ["lu", "qr"])
@pytest.mark.parametrize("mode", [REDUCED, EXTENDED])
def test_newton_200bus_matches_oracle_newton(P, mode, solver):
    sys = gridgen.grid_200()
    x0 = gridgen.flat_state(sys, mode == EXTENDED)
    xo, hist = oracle.newton_dense(sys, x0, mode)
    assert hist[-1] <= 1e-10
    ctx = P.Context(sys, MNAME[mode])
    ctx.set_newton_solver(solver)
    x = cuda(x0)
    info = ctx.newton(x, tol=1e-10, max_iter=20)
    assert info["converged"] == 1 and info["max_mismatch"] <= 1e-10
    assert abs(info["iterations"] - (len(hist) - 1)) <= 1, (info, len(hist))
    # both iterate to max |F| <= 1e-10: the same solution to well within 1e-8
    assert np.max(np.abs(x.cpu().numpy() - xo)) <= 1e-8
    assert np.max(np.abs(oracle.residual(sys, x.cpu().numpy(), mode))) <= 1e-10


def test_newton_two_bus_closed_form(P):
    """Slack (V = 1, theta = 0) - lossless line (x = 0.1) - PQ load 0.5 + j0.2:
    V^2 = [1 - 2 Q x + sqrt((1 - 2 Q x)^2 - 4 x^2 (P^2 + Q^2))] / 2,
    sin theta = -P x / V."""
    sys = two_bus()
    ctx = P.Context(sys)
    x = cuda(gridgen.flat_state(sys))
    info = ctx.newton(x, tol=1e-13, max_iter=20)
    assert info["converged"] == 1
    Pl, Ql, xl = 0.5, 0.2, 0.1
    a = 1 - 2 * Ql * xl
    v2 = math.sqrt((a + math.sqrt(a * a - 4 * xl * xl * (Pl * Pl + Ql * Ql))) / 2)
    th2 = math.asin(-Pl * xl / v2)
    xs = x.cpu().numpy()
    assert abs(xs[3] - v2) <= 1e-12 and abs(xs[1] - th2) <= 1e-12


@pytest.mark.parametrize("solver", ["lu", "qr"])
def test_newton_batched_outages(P, solver):
    sys = gridgen.grid_200()
    x0 = gridgen.flat_state(sys)
    # outages for which the oracle's Newton converges (the grid stays solvable)
    outs = []
    for l in range(0, sys.n_branch, 7):
        xo, hist = oracle.newton_dense(with_outage(sys, l), x0, max_iter=12)
        if hist[-1] <= 1e-10:
            outs.append((l, xo))
        if len(outs) == 6:
            break
    assert len(outs) == 6
    ctx = P.Context([sys], instances=[(0, l) for l, _ in outs])
    ctx.set_newton_solver(solver)
    x = cuda(np.concatenate([x0] * len(outs)))
    info = ctx.newton(x, tol=1e-10, max_iter=20)
    assert info["converged"] == 1
    xs = x.cpu().numpy()
    for k, (l, xo) in enumerate(outs):
        assert np.max(np.abs(xs[ctx.x_off[k]:ctx.x_off[k + 1]] - xo)) <= 1e-8, l


def test_mismatch_norm_and_update(P):
    grids = [gridgen.synthetic_grid(300, 4), gridgen.grid_200()]
    ctx = P.Context(grids, instances=[(0, -1), (1, -1), (0, 5)])
    xs = [gridgen.perturbed_state(grids[g], k + 1) for k, g in enumerate((0, 1, 0))]
    x = cuda(np.concatenate(xs))
    F = ctx.residual(x)
    norms = ctx.mismatch_norm(F).cpu().numpy()
    Fh = F.cpu().numpy()
    for k in range(3):
        assert norms[k] == np.max(np.abs(Fh[ctx.f_off[k]:ctx.f_off[k + 1]]))
    # update: x - dx on the unknowns, in J's column order, as the oracle's Newton does
    rng = np.random.default_rng(3)
    dx = rng.standard_normal(ctx.dims.n_f)
    x2 = ctx.newton_update(x.clone(), cuda(dx)).cpu().numpy()
    for k, g in enumerate((0, 1, 0)):
        fm = oracle.Formulation(grids[g], REDUCED)
        n = grids[g].n_bus
        want = xs[k].copy()
        d = dx[ctx.f_off[k]:ctx.f_off[k + 1]]
        ok = fm.col_th >= 0
        want[np.arange(n)[ok]] -= d[fm.col_th[ok]]
        ok = fm.col_v >= 0
        want[n + np.arange(n)[ok]] -= d[fm.col_v[ok]]
        assert np.array_equal(x2[ctx.x_off[k]:ctx.x_off[k + 1]], want)


def _modes(sys, seed):
    rng = np.random.default_rng(seed)
    ng = sys.n_pv + 1
    return rng.integers(0, 3, ng).astype(np.uint8), rng.uniform(-0.5, 0.8, ng)


def test_generator_modes_match_oracle(P):
    """Extended formulation with generators held at reactive limits (F, J and the VJP), in a
    batch where every instance has its own modes."""
    grids = [gridgen.synthetic_grid(30, 7, n_branch=39, cluster=10), gridgen.grid_200()]
    inst = [(0, -1), (1, -1), (1, 11), (0, 4)]
    ctx = P.Context(grids, "extended", instances=inst)
    xs, modes, qlims = [], [], []
    for k, (g, _) in enumerate(inst):
        xs.append(gridgen.perturbed_state(grids[g], k + 1, True))
        m, q = _modes(grids[g], 20 + k)
        modes.append(m)
        qlims.append(q)
    assert ctx.dims.n_gen_inst == sum(m.shape[0] for m in modes)
    X = cuda(np.concatenate(xs))
    gm = torch.from_numpy(np.concatenate(modes)).cuda()
    gq = cuda(np.concatenate(qlims))
    F, V = ctx.eval(X, ctx.empty_f(), ctx.empty_vals(), gen_mode=gm, gen_qlim=gq)
    Fh, Vh = F.cpu().numpy(), V.cpu().numpy()
    v = gridgen.gaussian_cotangents(ctx.dims.n_f, 1)[0]
    gx = ctx.vjp(X, cuda(v), 1, want=("x",), gen_mode=gm, gen_qlim=gq)["x"][0].cpu().numpy()
    for k, (g, out) in enumerate(inst):
        sysk = with_outage(grids[g], out)
        f = Fh[ctx.f_off[k]:ctx.f_off[k + 1]]
        assert_tol(f, oracle.residual(sysk, xs[k], EXTENDED, gen_mode=modes[k], gen_qlim=qlims[k]), f"F {k}")
        assert_tol(Vh[ctx.nnz_off[k]:ctx.nnz_off[k + 1]],
                   oracle.jacobian(sysk, xs[k], EXTENDED, gen_mode=modes[k])[2], f"J {k}")
        vk = v[ctx.f_off[k]:ctx.f_off[k + 1]]
        assert_tol(gx[ctx.x_off[k]:ctx.x_off[k + 1]],
                   oracle.vjp(sysk, xs[k], vk, EXTENDED, gen_mode=modes[k])["x"], f"v^T J {k}")
    # without modes every generator is in voltage control: the held entries are explicit zeros
    F0, V0 = ctx.residual_jacobian(X)
    for k, (g, out) in enumerate(inst):
        sysk = with_outage(grids[g], out)
        assert_tol(V0[ctx.nnz_off[k]:ctx.nnz_off[k + 1]].cpu().numpy(),
                   oracle.jacobian(sysk, xs[k], EXTENDED)[2], f"J voltage control {k}")


def test_newton_with_reactive_limits_matches_oracle(P):
    sys = gridgen.grid_200()
    n = sys.n_bus
    ng = sys.n_pv + 1
    x0 = gridgen.flat_state(sys, True)
    xe, _ = oracle.newton_dense(sys, x0, EXTENDED)
    q0 = xe[2 * n:2 * n + ng]
    q_max = np.full(ng, 1e30)
    q_min = np.full(ng, -1e30)
    q_max[[2, 9, 21]] = q0[[2, 9, 21]] - 0.05
    q_min[[5, 30]] = q0[[5, 30]] + 0.05
    xo, mo, qo, ro = oracle.newton_qlim(sys, x0, q_min, q_max)
    ctx = P.Context(sys, "extended")
    x = cuda(x0)
    info, rounds, gm, gq = ctx.newton_qlim(x, cuda(q_min), cuda(q_max), tol=1e-10)
    assert info["converged"] == 1 and rounds == ro
    assert np.array_equal(gm.cpu().numpy(), mo)
    assert np.max(np.abs(x.cpu().numpy() - xo)) <= 1e-8
    held = mo != 0
    assert np.array_equal(gq.cpu().numpy()[held], qo[held])


def test_fast_decoupled_matches_oracle(P):
    """Fast decoupled iterations (B', B'' factored once) vs the oracle's, on the 200-bus case and on a
    batch of outage instances; the fixed point is the Newton solution."""
    sys = gridgen.grid_200()
    x0 = gridgen.flat_state(sys)
    xo, ho = oracle.fdlf(sys, x0)
    xn, _ = oracle.newton_dense(sys, x0)
    ctx = P.Context(sys)
    x = cuda(x0)
    info = ctx.fdlf(x, tol=1e-10, max_iter=100)
    assert info["converged"] == 1 and abs(info["iterations"] - (len(ho) - 1)) <= 1, (info, len(ho))
    xs = x.cpu().numpy()
    assert np.max(np.abs(xs - xo)) <= 1e-8 and np.max(np.abs(xs - xn)) <= 1e-8
    outs = []
    for l in range(3, sys.n_branch, 11):
        xl, hl = oracle.fdlf(with_outage(sys, l), x0, max_iter=60)
        if hl[-1] <= 1e-10:
            outs.append((l, xl))
        if len(outs) == 4:
            break
    ctxb = P.Context([sys], instances=[(0, l) for l, _ in outs])
    xb = cuda(np.concatenate([x0] * len(outs)))
    info = ctxb.fdlf(xb, tol=1e-10, max_iter=100)
    assert info["converged"] == 1
    xbs = xb.cpu().numpy()
    for k, (l, xl) in enumerate(outs):
        assert np.max(np.abs(xbs[ctxb.x_off[k]:ctxb.x_off[k + 1]] - xl)) <= 1e-8, l


def _constructed(n_bus, seed):
    """A grid of the paper's shape with a known solution: injections (the oracle's) equal to the
    network's own flows at gridgen.target_state."""
    g = gridgen.grid_70k() if n_bus == 70000 else gridgen.synthetic_grid(n_bus, seed)
    th, V = gridgen.target_state(g, seed + 1)
    z = np.zeros(g.n_bus)
    fp, fq = oracle.bus_mismatch(g, th, V, p_inj=z, q_inj=z)
    return gridgen.with_injections(g, fp, fq, V), np.concatenate([th, V])


@pytest.mark.parametrize("n_bus,solver", [(70000, "lu"), (25000, "lu"), (10000, "qr")])
def test_newton_constructed_grid_from_flat_start(P, n_bus, solver):
    """Flat-start Newton (reduced formulation) on the constructed case of the 70k grid (the
    paper's test-system size, Sec. IV-A) and of 25k and 10k grids: converged, the oracle's
    residual at the GPU's solution within 1e-8, and the solution is the point the case was
    built around."""
    sys, xs = _constructed(n_bus, 2500)
    ctx = P.Context(sys)
    ctx.set_newton_solver(solver)
    x = cuda(gridgen.flat_state(sys))
    info = ctx.newton(x, tol=1e-9, max_iter=20)
    assert info["converged"] == 1 and info["max_mismatch"] <= 1e-9, info
    assert info["iterations"] <= 12, info
    xg = x.cpu().numpy()
    assert np.max(np.abs(oracle.residual(sys, xg))) <= 1e-8
    assert np.max(np.abs(xg - xs)) <= 1e-7
    ctx.close()
