"""The allocation-free entry point pf_residual_jacobian_static, through the C ABI.

It is for callers that cannot allocate device memory when they evaluate (it
uses a static device array as scratch instead of memory from cudaMalloc).
It runs the same kernels as pf_residual_jacobian, so on the same context,
state and tuning its F and J must equal pf_residual_jacobian's bit for bit,
on two calls in a row (the second call reuses the array the first one left
behind), and match the oracle within the parity tolerance.  It must not
change the device's free memory, must accept a context of exactly the
static array's capacity (a batch with outages, under a persistent grid and
split rounds), and must refuse a larger one.  Collected last so that a run
stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import gridgen
import oracle
from tests.gpu_common import assert_tol

pytestmark = pytest.mark.gpu

CAPACITY = 1 << 18          # instance-buses the static scratch holds


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2011_11880_gb300 as p
    return p


def call_static(ctx, x, F, V):
    from paper_2011_11880_gb300 import _lib
    lib = _lib.load()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.pf_residual_jacobian_static(ctx._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(F.data_ptr()),
                                         ctypes.c_void_p(V.data_ptr()), s)
    msg = lib.pf_last_error()
    return rc, (msg or b"").decode()


@pytest.mark.parametrize("mode", ["reduced", "extended"])
def test_static_scratch_matches_pf_residual_jacobian(P, mode):
    sys_ = gridgen.synthetic_grid(3000, 13, end_g_frac=0.1, xfmr_frac=0.2, shift_frac=0.2)
    ext = mode == "extended"
    ctx = P.Context(sys_, mode)
    for k in (1, 2):                              # two calls in a row, different states
        x_np = gridgen.perturbed_state(sys_, k, ext)
        x = torch.from_numpy(x_np).cuda()
        F_ref, V_ref = ctx.residual_jacobian(x)
        F = torch.full_like(F_ref, np.nan)
        V = torch.full_like(V_ref, np.nan)
        rc, msg = call_static(ctx, x, F, V)
        assert rc == 0, msg
        torch.cuda.synchronize()
        assert torch.equal(F, F_ref), f"F call {k} differs from pf_residual_jacobian"
        assert torch.equal(V, V_ref), f"J call {k} differs from pf_residual_jacobian"
        if k == 1:
            om = oracle.EXTENDED if ext else oracle.REDUCED
            assert_tol(F.cpu().numpy(), oracle.residual(sys_, x_np, om), f"F vs oracle ({mode})")
            assert_tol(V.cpu().numpy(), oracle.jacobian(sys_, x_np, om)[2], f"J vs oracle ({mode})")
    ctx.check_device()
    ctx.close()


def test_static_scratch_allocates_nothing(P):
    sys_ = gridgen.synthetic_grid(2000, 5)
    ctx = P.Context(sys_)
    x = torch.from_numpy(gridgen.perturbed_state(sys_, 3)).cuda()
    F, V = ctx.empty_f(), ctx.empty_vals()
    assert call_static(ctx, x, F, V)[0] == 0      # the first call on the device resolves the array
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(5):
        rc, msg = call_static(ctx, x, F, V)
        assert rc == 0, msg
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0, "free device memory changed across static calls"
    assert torch.cuda.memory_reserved() == reserved0
    ctx.close()


def test_static_scratch_full_capacity_batch_with_outages(P):
    # 256 instances of a 1,024-bus grid: exactly the capacity of the static array,
    # every instance with its own branch outage (the masked kernels), evaluated under
    # a persistent grid and under split rounds
    g = gridgen.synthetic_grid(1024, 21)
    rng = np.random.default_rng(7)
    outages = rng.integers(0, g.br_from.shape[0], size=256)
    ctx = P.Context([g], instances=[(0, int(o)) for o in outages])
    assert ctx.dims.n_bus_inst == CAPACITY
    x_np = np.concatenate([gridgen.perturbed_state(g, 100 + k) for k in range(256)])
    x = torch.from_numpy(x_np).cuda()
    for tuning in ((32, 12, 0), (64, 0, 1)):
        ctx.set_tuning(*tuning)
        F_ref, V_ref = ctx.residual_jacobian(x)
        for call in range(2):
            F = torch.full_like(F_ref, np.nan)
            V = torch.full_like(V_ref, np.nan)
            rc, msg = call_static(ctx, x, F, V)
            assert rc == 0, msg
            torch.cuda.synchronize()
            assert torch.equal(F, F_ref), f"F differs (tuning {tuning}, call {call})"
            assert torch.equal(V, V_ref), f"J differs (tuning {tuning}, call {call})"
        ctx.check_device()
    # one instance against the oracle with its outage applied
    k = 17
    gk = g.copy()
    gk.br_status = gk.br_status.copy()
    gk.br_status[outages[k]] = 0
    xk = x_np[k * 2 * 1024:(k + 1) * 2 * 1024]
    f0, f1 = ctx.f_off[k], ctx.f_off[k + 1]
    assert_tol(F[f0:f1].cpu().numpy(), oracle.residual(gk, xk), "F vs oracle (outage instance)")
    ctx.close()


def test_static_scratch_rejects_oversized_context(P):
    g = gridgen.synthetic_grid(1000, 4)
    ctx = P.Context([g], instances=[(0, -1)] * 300)        # 300,000 instance-buses > 2^18
    x = torch.zeros(ctx.dims.n_x, dtype=torch.float64, device="cuda")
    F, V = ctx.empty_f(), ctx.empty_vals()
    rc, msg = call_static(ctx, x, F, V)
    assert rc == 5 and "static scratch holds at most 262144" in msg, (rc, msg)
    ctx.close()
