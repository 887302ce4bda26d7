"""Failure paths of the build, injected on the host (no GPU fault): with
PF_FAIL_ALLOC=<n> the n-th device allocation of a build reports failure.
Every such build must return PF_ERR_OOM, free what it had allocated, and leave
the library usable.  GPU only (the allocations are real up to the failing one)."""
import numpy as np
import pytest
import torch

import gridgen
import oracle
from tests.gpu_common import assert_tol

pytestmark = pytest.mark.gpu
PF_ERR_OOM = 2


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2011_11880_gb300 as p
    return p


@pytest.mark.parametrize("batched", [False, True])
def test_every_allocation_failure_of_a_build(P, monkeypatch, batched):
    grids = [gridgen.grid_200(), gridgen.synthetic_grid(30, 7, n_branch=39, cluster=10)]
    build = (lambda: P.Context(grids, instances=[(0, -1), (1, 4), (0, 9)])) if batched else \
            (lambda: P.Context(grids[0]))
    ctx = build()                                 # warm: the CUDA context and the library's statics
    ctx.close()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    for n in range(10000):
        monkeypatch.setenv("PF_FAIL_ALLOC", str(n))
        try:
            ctx = build()
        except P.PFError as e:
            assert e.code == PF_ERR_OOM, (n, e)
            failures += 1
            continue
        ctx.close()                               # n is past the build's last allocation
        break
    assert failures > 20                          # every allocation of the build was made to fail
    monkeypatch.delenv("PF_FAIL_ALLOC")
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert abs(free1 - free0) <= 8 << 20, (free0, free1)   # nothing left allocated
    # and the library still works
    ctx = P.Context(grids[0])
    x = gridgen.perturbed_state(grids[0], 2)
    F, J = ctx.residual_jacobian(torch.from_numpy(x).cuda())
    assert_tol(F.cpu().numpy(), oracle.residual(grids[0], x), "F after the failures")
    assert_tol(J.cpu().numpy(), oracle.jacobian(grids[0], x)[2], "J after the failures")
    ctx.check_device()
