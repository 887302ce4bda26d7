"""The allocation-free entry point pf_residual_jacobian_static, through the C ABI.

It is for callers that cannot allocate device memory when they evaluate (it
uses a static device array as scratch instead of memory from cudaMalloc).
Its F and J must equal those of pf_residual_jacobian on the same context
within the parity tolerance, on two calls in a row (the second call reuses
the array the first one left behind), and it must refuse a context larger
than its static scratch.  Collected last so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import gridgen
from tests.gpu_common import assert_tol

pytestmark = pytest.mark.gpu


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
        x = torch.from_numpy(gridgen.perturbed_state(sys_, k, ext)).cuda()
        F_ref, V_ref = ctx.residual_jacobian(x)
        F = torch.full_like(F_ref, np.nan)
        V = torch.full_like(V_ref, np.nan)
        rc, msg = call_static(ctx, x, F, V)
        assert rc == 0, msg
        torch.cuda.synchronize()
        assert_tol(F.cpu().numpy(), F_ref.cpu().numpy(), f"F call {k}")
        assert_tol(V.cpu().numpy(), V_ref.cpu().numpy(), f"J call {k}")
    ctx.check_device()
    ctx.close()


def test_static_scratch_rejects_oversized_context(P):
    g = gridgen.synthetic_grid(1000, 4)
    ctx = P.Context([g], instances=[(0, -1)] * 300)        # 300,000 instance-buses > 2^18
    x = torch.zeros(ctx.dims.n_x, dtype=torch.float64, device="cuda")
    F, V = ctx.empty_f(), ctx.empty_vals()
    rc, msg = call_static(ctx, x, F, V)
    assert rc == 5 and "static scratch holds at most 262144" in msg, (rc, msg)
    ctx.close()
