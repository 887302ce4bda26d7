"""The batched and adjoint workloads at their full sizes, launched the way a
caller runs them (one context, autotuned, replayed from a captured CUDA
graph), checked against the CPU oracle on sampled instances / cotangents and
by properties that hold at any size.  GPU only.

  * 2,048 instances of a 2,000-bus grid + 256 of a 10,000-bus grid, one
    seeded branch outage each;
  * the 70,000-bus grid with 64 Gaussian cotangents through the
    torch.autograd.Function;
  * 4,096 instances of their own grids (500 to 20,000 buses, log-uniform)
    with perturbed injections: F + J, then the VJP with F as cotangent, in
    one captured iteration.
"""
import numpy as np
import pytest
import torch

import gridgen
import oracle
from tests.gpu_common import assert_tol, with_outage

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2011_11880_gb300 as p
    return p


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def captured(fn, stream):
    """fn() once, then captured into a CUDA graph and replayed once."""
    with torch.cuda.stream(stream):
        fn()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            fn()
        g.replay()
    torch.cuda.synchronize()
    return g


def test_contingency_batch_full_size(P):
    grids, insts = gridgen.contingency_batch()
    assert len(insts) == 2304
    ctx = P.Context(grids, instances=[(i.grid, i.outage) for i in insts])
    X = cuda(np.concatenate([i.x for i in insts]))
    F, V = ctx.empty_f(), ctx.empty_vals()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx.autotune(X, F, V, stream=s)
    captured(lambda: ctx.residual_jacobian(X, F, V, stream=s), s)
    assert torch.isfinite(F).all() and torch.isfinite(V).all()
    Fh, Vh = F.cpu().numpy(), V.cpu().numpy()
    # patterns of both grids, bit-exact
    for gi, sys in enumerate(grids):
        rp, ci = ctx.pattern(gi)
        rpo, cio, _ = oracle.jacobian(sys, gridgen.flat_state(sys))
        assert np.array_equal(rp, rpo) and np.array_equal(ci, cio)
    # F of every instance (its outage applied) against the oracle
    for k, ins in enumerate(insts):
        f = Fh[ctx.f_off[k]:ctx.f_off[k + 1]]
        assert_tol(f, oracle.residual(with_outage(grids[ins.grid], ins.outage), ins.x), f"instance {k} F")
    rng = np.random.default_rng(33)
    sample = sorted({0, 1, 1023, 2047, 2048, 2175, 2303, *rng.integers(0, 2304, 5).tolist()})
    for k in sample:
        ins = insts[k]
        sys = with_outage(grids[ins.grid], ins.outage)
        f = Fh[ctx.f_off[k]:ctx.f_off[k + 1]]
        vals = Vh[ctx.nnz_off[k]:ctx.nnz_off[k + 1]]
        assert_tol(f, oracle.residual(sys, ins.x), f"instance {k} F")
        assert_tol(vals, oracle.jacobian(sys, ins.x)[2], f"instance {k} J")
    # the masked batch gives the bits of a plain single-instance context of the outaged grid
    for k in (5, 2200):
        ins = insts[k]
        one = P.Context(with_outage(grids[ins.grid], ins.outage))
        f1, v1 = one.residual_jacobian(cuda(ins.x))
        assert torch.equal(f1, F[ctx.f_off[k]:ctx.f_off[k + 1]])
        assert torch.equal(v1, V[ctx.nnz_off[k]:ctx.nnz_off[k + 1]])
    ctx.check_device()


def test_adjoint_70k_64_cotangents(P):
    from paper_2011_11880_gb300 import residual
    sys = gridgen.grid_70k()
    ctx = P.Context(sys)
    d = ctx.dims
    B = 64
    xn = gridgen.perturbed_state(sys, 1)
    Vn = gridgen.gaussian_cotangents(d.n_f, B)                 # seeds 4000 + k
    x = cuda(xn)
    r, xr, bc, tap = (cuda(a) for a in (sys.br_r, sys.br_x, sys.br_b, sys.br_tap))
    p0, q0 = oracle.net_injections(sys)
    pin, qin = cuda(p0), cuda(q0)
    leaves = [t.unsqueeze(0).expand(B, -1).requires_grad_() for t in (x, pin, qin, r, xr, bc, tap)]
    Fb = residual(ctx, *leaves)
    assert Fb.shape == (B, d.n_f)
    grads = torch.autograd.grad(Fb, leaves, grad_outputs=cuda(Vn))
    gx, gp, gq, gr, gxr, gb, gt = (g.cpu().numpy() for g in grads)
    for c in (0, 21, 63):
        go = oracle.vjp(sys, xn, Vn[c])
        assert_tol(gx[c], go["x"], f"dx cot {c}")
        assert_tol(gp[c], go["p_inj"], f"dP_inj cot {c}")
        assert_tol(gq[c], go["q_inj"], f"dQ_inj cot {c}")
        assert_tol(gr[c], go["r"], f"dr cot {c}")
        assert_tol(gxr[c], go["reac"], f"dx_branch cot {c}")
        assert_tol(gb[c], go["b"], f"db_c cot {c}")
        assert_tol(gt[c], go["tap"], f"dtap cot {c}")
    # every cotangent of the batch equals its own single-cotangent call, bit for bit
    V = cuda(Vn).reshape(-1)
    gall = ctx.vjp(x, V, B)
    for c in range(B):
        g1 = ctx.vjp(x, cuda(Vn[c]), 1)
        for k in g1:
            assert torch.equal(g1[k][0], gall[k][c]), (k, c)
    # central differences of the GPU forward along random directions of x
    rng = np.random.default_rng(7)
    h = 1e-7
    for c in (3, 40):
        dvec = rng.standard_normal(d.n_x)
        Fp = ctx.residual(cuda(xn + h * dvec)).cpu().numpy()
        Fm = ctx.residual(cuda(xn - h * dvec)).cpu().numpy()
        fd = Vn[c] @ (Fp - Fm) / (2 * h)
        an = gall["x"][c].cpu().numpy() @ dvec
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (c, fd, an)
    ctx.check_device()


def test_mixed_batch_full_size_iteration(P):
    grids, insts = gridgen.mixed_batch()
    assert len(insts) == 4096
    ctx = P.Context(grids, instances=[(k, -1) for k in range(len(grids))])
    d = ctx.dims
    X = cuda(np.concatenate([i.x for i in insts]))
    Pi = cuda(np.concatenate([i.p_inj for i in insts]))
    Qi = cuda(np.concatenate([i.q_inj for i in insts]))
    F, V = ctx.empty_f(), ctx.empty_vals()
    G = torch.empty(d.n_x, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx.autotune(X, F, V, stream=s)

    def iteration():
        ctx.eval(X, F, V, stream=s, p_inj=Pi, q_inj=Qi)
        g = ctx.vjp(X, F, 1, want=("x",), stream=s, p_inj=Pi, q_inj=Qi)["x"]
        G.copy_(g[0])

    captured(iteration, s)
    assert torch.isfinite(F).all() and torch.isfinite(V).all() and torch.isfinite(G).all()
    Fh, Vh, Gh = F.cpu().numpy(), V.cpu().numpy(), G.cpu().numpy()
    # F of every instance against the oracle (with its injection overrides)
    for k, (ins, sys) in enumerate(zip(insts, grids)):
        f = Fh[ctx.f_off[k]:ctx.f_off[k + 1]]
        assert_tol(f, oracle.residual(sys, ins.x, p_inj=ins.p_inj, q_inj=ins.q_inj), f"instance {k} F")
    sizes = np.array([g.n_bus for g in grids])
    rng = np.random.default_rng(55)
    sample = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 0, 4095, *rng.integers(0, 4096, 4).tolist()})
    for k in sample:
        ins, sys = insts[k], grids[k]
        f = Fh[ctx.f_off[k]:ctx.f_off[k + 1]]
        assert_tol(f, oracle.residual(sys, ins.x, p_inj=ins.p_inj, q_inj=ins.q_inj), f"instance {k} F")
        assert_tol(Vh[ctx.nnz_off[k]:ctx.nnz_off[k + 1]], oracle.jacobian(sys, ins.x)[2], f"instance {k} J")
        go = oracle.vjp(sys, ins.x, f)
        assert_tol(Gh[ctx.x_off[k]:ctx.x_off[k + 1]], go["x"], f"instance {k} J^T F")
    ctx.check_device()
