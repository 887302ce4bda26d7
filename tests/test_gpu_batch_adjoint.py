"""Batched instances (outage masks, injection overrides, uneven grid sizes)
and the adjoint kernels vs the CPU oracle.  GPU only."""
import numpy as np
import pytest
import torch

import gridgen
import oracle
from oracle import REDUCED, EXTENDED
from tests.gpu_common import assert_tol, edge_grid, star_grid, state, three_bus, with_outage

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


@pytest.mark.parametrize("mode", [REDUCED, EXTENDED])
def test_batch_outages_uneven_sizes(P, mode):
    grids = [gridgen.synthetic_grid(200, 1), gridgen.synthetic_grid(1200, 2), three_bus()]
    rng = np.random.default_rng(5)
    inst = []
    for k in range(40):
        g = [0, 1, 2][k % 3]
        out = int(rng.integers(-1, grids[g].n_branch))
        inst.append((g, out))
    ctx = P.Context(grids, MNAME[mode], instances=inst)
    xs = [state(grids[g], 1 + k, mode == EXTENDED) for k, (g, _) in enumerate(inst)]
    x = cuda(np.concatenate(xs))
    F, v = ctx.residual_jacobian(x)
    F, v = F.cpu().numpy(), v.cpu().numpy()
    for k, (g, out) in enumerate(inst):
        s = with_outage(grids[g], out)
        Fk = F[ctx.f_off[k]:ctx.f_off[k + 1]]
        vk = v[ctx.nnz_off[k]:ctx.nnz_off[k + 1]]
        assert_tol(Fk, oracle.residual(s, xs[k], mode), f"inst {k} F")
        assert_tol(vk, oracle.jacobian(s, xs[k], mode)[2], f"inst {k} J")
    # the pattern of a grid is independent of the outage
    for g in range(3):
        rp, ci = ctx.pattern(g)
        rpo, cio, _ = oracle.jacobian(grids[g], state(grids[g], 0, mode == EXTENDED), mode)
        assert np.array_equal(rp, rpo) and np.array_equal(ci, cio)
    ctx.check_device()


def test_batch_without_outage_equals_single(P):
    """An instance with no outage in a masked batch gives the same bits as a plain build."""
    g = gridgen.synthetic_grid(500, 9)
    ctx1 = P.Context(g)
    ctxb = P.Context([g], instances=[(0, 3), (0, -1)])
    xn = state(g, 2)
    F1, v1 = ctx1.residual_jacobian(cuda(xn))
    Fb, vb = ctxb.residual_jacobian(cuda(np.concatenate([xn, xn])))
    n_f, nnz = ctx1.dims.n_f, ctx1.dims.nnz
    assert torch.equal(F1, Fb[n_f:]) and torch.equal(v1, vb[nnz:])


def test_status_and_injection_overrides(P):
    grids = [gridgen.synthetic_grid(300, 4), star_grid(300)]
    inst = [(0, -1), (1, -1), (0, 5)]
    ctx = P.Context(grids, instances=inst)
    d = ctx.dims
    rng = np.random.default_rng(7)
    xs = [state(grids[g], 3 + k) for k, (g, _) in enumerate(inst)]
    status = (rng.random(d.n_branch_inst) > 0.1).astype(np.uint8)
    pi, qi = [], []
    for g, _ in inst:
        p0, q0 = oracle.net_injections(grids[g])
        pi.append(p0 * rng.uniform(0.5, 1.5, p0.shape))
        qi.append(q0 * rng.uniform(0.8, 1.2))
    F, v = ctx.eval(cuda(np.concatenate(xs)), ctx.empty_f(), ctx.empty_vals(), status=cuda(status),
                    p_inj=cuda(np.concatenate(pi)), q_inj=cuda(np.concatenate(qi)))
    F, v = F.cpu().numpy(), v.cpu().numpy()
    bo = 0
    for k, (g, out) in enumerate(inst):
        s = grids[g].copy()
        m = grids[g].n_branch
        s.br_status = (grids[g].br_status * status[bo:bo + m]).astype(np.uint8)
        if out >= 0:
            s.br_status[out] = 0
        bo += m
        assert_tol(F[ctx.f_off[k]:ctx.f_off[k + 1]], oracle.residual(s, xs[k], REDUCED, p_inj=pi[k], q_inj=qi[k]))
        assert_tol(v[ctx.nnz_off[k]:ctx.nnz_off[k + 1]], oracle.jacobian(s, xs[k])[2])


# ---------------------------------------------------------------------------
# adjoint
# ---------------------------------------------------------------------------

def check_vjp(P, sys, mode, n_cot=3, outage=-1, seed=0):
    ctx = P.Context([sys], MNAME[mode], instances=[(0, outage)])
    xn = state(sys, 2, mode == EXTENDED)
    V = gridgen.gaussian_cotangents(ctx.dims.n_f, n_cot, seed=4000 + seed)
    g = ctx.vjp(cuda(xn), cuda(V.reshape(-1)), n_cot=n_cot)
    s = with_outage(sys, outage)
    for c in range(n_cot):
        go = oracle.vjp(s, xn, V[c], mode)
        for k_gpu, k_or in (("x", "x"), ("p_inj", "p_inj"), ("q_inj", "q_inj"), ("br_r", "r"),
                            ("br_x", "reac"), ("br_b", "b"), ("br_tap", "tap")):
            assert_tol(g[k_gpu][c].cpu().numpy(), go[k_or], f"{k_gpu} cot {c}")
    ctx.check_device()


@pytest.mark.parametrize("mode", [REDUCED, EXTENDED])
def test_vjp_matches_oracle(P, mode):
    for sys in (three_bus(), gridgen.synthetic_grid(30, 7, n_branch=39, end_g_frac=0.2, xfmr_frac=0.3,
                                                    shift_frac=0.3, cluster=10), edge_grid()):
        check_vjp(P, sys, mode)


def test_vjp_big_bus_and_outage(P):
    check_vjp(P, star_grid(1300), REDUCED, n_cot=2)
    check_vjp(P, gridgen.grid_200(), REDUCED, n_cot=2, outage=17)


def test_vjp_against_gpu_central_differences(P):
    """v^T dF/dx from the adjoint kernel vs central differences (h = 1e-7) of the GPU forward."""
    sys = gridgen.grid_200()
    ctx = P.Context(sys)
    xn = state(sys, 1)
    v = gridgen.gaussian_cotangents(ctx.dims.n_f, 1)[0]
    g = ctx.vjp(cuda(xn), cuda(v), want=("x",))["x"][0].cpu().numpy()
    h = 1e-7
    for j in range(0, xn.shape[0], 13):
        xp, xm = xn.copy(), xn.copy()
        xp[j] += h
        xm[j] -= h
        d = (v @ ctx.residual(cuda(xp)).cpu().numpy() - v @ ctx.residual(cuda(xm)).cpu().numpy()) / (2 * h)
        assert abs(d - g[j]) <= 1e-5 * max(1.0, abs(d)), (j, d, g[j])


def test_autograd_function_single_and_batched(P):
    from paper_2011_11880_gb300 import residual
    sys = gridgen.synthetic_grid(120, 3, end_g_frac=0.2)
    ctx = P.Context(sys)
    xn = state(sys, 4)
    x = cuda(xn).requires_grad_()
    r = cuda(sys.br_r).requires_grad_()
    tap = cuda(sys.br_tap).requires_grad_()
    F = residual(ctx, x, br_r=r, br_tap=tap)
    assert_tol(F.detach().cpu().numpy(), oracle.residual(sys, xn), "autograd forward")
    v = gridgen.gaussian_cotangents(ctx.dims.n_f, 1)[0]
    gx, gr, gt = torch.autograd.grad(F, (x, r, tap), grad_outputs=cuda(v))
    go = oracle.vjp(sys, xn, v)
    assert_tol(gx.cpu().numpy(), go["x"], "autograd dx")
    assert_tol(gr.cpu().numpy(), go["r"], "autograd dr")
    assert_tol(gt.cpu().numpy(), go["tap"], "autograd dtap")
    # batch of cotangents: inputs expanded with stride 0
    B = 5
    V = gridgen.gaussian_cotangents(ctx.dims.n_f, B, seed=77)
    xb = x.detach().unsqueeze(0).expand(B, -1).requires_grad_()
    rb = r.detach().unsqueeze(0).expand(B, -1).requires_grad_()
    Fb = residual(ctx, xb, br_r=rb)
    assert Fb.shape == (B, ctx.dims.n_f)
    gxb, grb = torch.autograd.grad(Fb, (xb, rb), grad_outputs=cuda(V))
    for c in range(B):
        goc = oracle.vjp(sys, xn, V[c])
        assert_tol(gxb[c].cpu().numpy(), goc["x"], f"batched dx {c}")
        assert_tol(grb[c].cpu().numpy(), goc["r"], f"batched dr {c}")


def test_many_tiny_grids_in_one_batch(P):
    """2,000 instances of 2- to 40-bus grids (rounds mostly partly filled), each its own grid."""
    rng = np.random.default_rng(8)
    grids = [gridgen.synthetic_grid(int(n), 100 + k) for k, n in enumerate(rng.integers(2, 41, 2000))]
    ctx = P.Context(grids, instances=[(k, -1) for k in range(len(grids))])
    xs = [gridgen.perturbed_state(g, k + 1) for k, g in enumerate(grids)]
    F, V = ctx.residual_jacobian(cuda(np.concatenate(xs)))
    Fh, Vh = F.cpu().numpy(), V.cpu().numpy()
    for k in list(range(0, 2000, 97)) + [1999]:
        assert_tol(Fh[ctx.f_off[k]:ctx.f_off[k + 1]], oracle.residual(grids[k], xs[k]), f"grid {k} F")
        assert_tol(Vh[ctx.nnz_off[k]:ctx.nnz_off[k + 1]], oracle.jacobian(grids[k], xs[k])[2], f"grid {k} J")
    ctx.check_device()


@pytest.mark.parametrize("mode", [REDUCED, EXTENDED])
def test_every_branch_out_of_service(P, mode):
    """Degenerate network: no branch in service (F is the injections and shunts alone), built
    plain and as a masked batch instance."""
    sys = gridgen.grid_200()
    dead = sys.copy()
    dead.br_status = np.zeros_like(sys.br_status)
    x = gridgen.perturbed_state(sys, 3, mode == EXTENDED)
    F0 = oracle.residual(dead, x, mode)
    J0 = oracle.jacobian(dead, x, mode)[2]
    ctx = P.Context(dead, MNAME[mode])
    F, V = ctx.residual_jacobian(cuda(x))
    assert_tol(F.cpu().numpy(), F0, "F")
    assert_tol(V.cpu().numpy(), J0, "J")
    status = torch.zeros(sys.n_branch, dtype=torch.uint8, device="cuda")
    ctx2 = P.Context(sys, MNAME[mode])
    F2, V2 = ctx2.eval(cuda(x), ctx2.empty_f(), ctx2.empty_vals(), status=status)
    assert_tol(F2.cpu().numpy(), F0, "F masked")
    assert_tol(V2.cpu().numpy(), J0, "J masked")


def test_host_buffers_pipelined_batch(P):
    """pf_residual_jacobian_host on a batch (pipelined over chunks of instances) gives the
    device path's bits, from pageable and from page-locked host buffers."""
    grids = [gridgen.synthetic_grid(300, 2), gridgen.synthetic_grid(1100, 3), gridgen.grid_200()]
    rng = np.random.default_rng(12)
    inst = [(int(g), int(rng.integers(-1, 200))) for g in rng.integers(0, 3, 21)]
    ctx = P.Context(grids, instances=inst)
    xn = np.concatenate([gridgen.perturbed_state(grids[g], k + 1) for k, (g, _) in enumerate(inst)])
    F_d, v_d = ctx.residual_jacobian(cuda(xn))
    F_d, v_d = F_d.cpu().numpy(), v_d.cpu().numpy()
    for pinned in (False, True):
        if pinned:
            xh = torch.from_numpy(xn).pin_memory().numpy()
            F_h = torch.empty(ctx.dims.n_f, dtype=torch.float64).pin_memory().numpy()
            v_h = torch.empty(ctx.dims.nnz, dtype=torch.float64).pin_memory().numpy()
        else:
            xh, F_h, v_h = xn.copy(), np.empty(ctx.dims.n_f), np.empty(ctx.dims.nnz)
        ctx.residual_jacobian_host(xh, F_h, v_h)
        assert np.array_equal(F_h, F_d) and np.array_equal(v_h, v_d), pinned
        F_only = np.empty(ctx.dims.n_f)
        ctx.residual_jacobian_host(xh, F_only, None)
        assert np.array_equal(F_only, F_d)


@pytest.mark.parametrize("mode", [REDUCED, EXTENDED])
def test_large_bus_under_outages_and_modes(P, mode):
    """The warp-per-bus kernel (a hub with 1,500 neighbours) under branch outages, with a PV
    unit on the hub held at a reactive limit in the extended formulation."""
    sys = star_grid(1500)
    sys.pv_bus = sys.pv_bus.copy()
    sys.pv_bus[0] = 0                                   # a generator on the hub
    inst = [(0, -1), (0, 0), (0, 1), (0, 1503)]          # outages of hub branches and of a parallel one
    ctx = P.Context([sys], MNAME[mode], instances=inst)
    xs = [gridgen.perturbed_state(sys, k + 1, mode == EXTENDED) for k in range(len(inst))]
    ov = {}
    gm = None
    if mode == EXTENDED:
        ng = sys.n_pv + 1
        gm = np.zeros(ng, np.uint8)
        gm[0] = 1
        gq = np.full(ng, 0.25)
        ov = dict(gen_mode=torch.from_numpy(np.tile(gm, len(inst))).cuda(), gen_qlim=cuda(np.tile(gq, len(inst))))
    F, V = ctx.eval(cuda(np.concatenate(xs)), ctx.empty_f(), ctx.empty_vals(), **ov)
    Fh, Vh = F.cpu().numpy(), V.cpu().numpy()
    for k, (_, out) in enumerate(inst):
        sk = with_outage(sys, out)
        kw = dict(gen_mode=gm, gen_qlim=np.full(sys.n_pv + 1, 0.25)) if mode == EXTENDED else {}
        assert_tol(Fh[ctx.f_off[k]:ctx.f_off[k + 1]], oracle.residual(sk, xs[k], mode, **kw), f"F {k}")
        jkw = dict(gen_mode=gm) if mode == EXTENDED else {}
        assert_tol(Vh[ctx.nnz_off[k]:ctx.nnz_off[k + 1]], oracle.jacobian(sk, xs[k], mode, **jkw)[2], f"J {k}")
    ctx.check_device()


@pytest.mark.parametrize("mode", [REDUCED, EXTENDED])
def test_branchless_buses_and_smallest_grids(P, mode):
    """Degenerate grids: buses without any branch (a grid whose only branch is taken out by
    the outage has no pair at all), a two-bus grid of a slack and a PV unit (one row in the
    reduced formulation), alone and in one batch with a normal grid.  (A one-bus grid is
    refused by pf_build's host validation.)"""
    bare = gridgen.PowerSystem.build(2, branches=[(0, 1, 0.01, 0.1, 0.02)], slack=(0, 1.02, 0.1),
                                     pvs=[(1, 0.2, 1.01)], shunts=[(0, 0.01, 0.2)])
    islands = gridgen.PowerSystem.build(4, branches=[(0, 1, 0.01, 0.1, 0.02)], loads=[(2, 0.3, 0.1), (3, 0.2, 0.0)],
                                        slack=(0, 1.0, 0.0), shunts=[(3, 0.0, 0.1)])
    grids = [bare, islands, three_bus()]
    ext = mode == EXTENDED
    for g in grids[:2]:
        ctx = P.Context(g, "extended" if ext else "reduced")
        x_np = gridgen.perturbed_state(g, 2, ext)
        F, v = ctx.residual_jacobian(torch.from_numpy(x_np).cuda())
        rp, ci, jo = oracle.jacobian(g, x_np, mode)
        assert F.numel() == len(rp) - 1 and v.numel() == len(ci)
        assert_tol(F.cpu().numpy(), oracle.residual(g, x_np, mode), "F degenerate")
        assert_tol(v.cpu().numpy(), jo, "J degenerate")
        ctx.check_device()
    inst = [(0, -1), (1, -1), (2, 3), (0, 0), (1, 0)]
    ctx = P.Context(grids, "extended" if ext else "reduced", instances=inst)
    xs = [gridgen.perturbed_state(grids[g], k + 1, ext) for k, (g, _) in enumerate(inst)]
    x = torch.from_numpy(np.concatenate(xs)).cuda()
    F, v = ctx.residual_jacobian(x)
    fo, vo = ctx.f_off, ctx.nnz_off
    for k, (g, out) in enumerate(inst):
        sk = grids[g] if out < 0 else with_outage(grids[g], out)
        assert_tol(F[fo[k]:fo[k + 1]].cpu().numpy(), oracle.residual(sk, xs[k], mode), f"F inst {k}")
        assert_tol(v[vo[k]:vo[k + 1]].cpu().numpy(), oracle.jacobian(sk, xs[k], mode)[2], f"J inst {k}")
    ctx.check_device()
