"""Shared helpers of the GPU parity tests (CUDA path vs the CPU oracle)."""
import numpy as np

import gridgen
import oracle

RTOL = 1e-12   # parity tolerance: |gpu - oracle| <= 1e-10 + 1e-12 |oracle|
ATOL = 1e-10


def assert_tol(got, want, what=""):
    got = np.asarray(got)
    want = np.asarray(want)
    assert got.shape == want.shape, (what, got.shape, want.shape)
    err = np.abs(got - want)
    bound = ATOL + RTOL * np.abs(want)
    bad = ~(err <= bound)
    if bad.any():
        i = int(np.argmax(np.where(bad, err - bound, -np.inf)))
        raise AssertionError(f"{what}: {int(bad.sum())}/{got.size} outside tolerance; worst index {i}: "
                             f"gpu {got.flat[i]!r} oracle {want.flat[i]!r}")


def three_bus():
    return gridgen.PowerSystem.build(
        3,
        branches=[
            (0, 1, 0.01, 0.08, 0.04),
            (1, 2, 0.02, 0.12, 0.03, 1.0, 0.0, 0.002, 0.003),
            (2, 0, 0.015, 0.10, 0.0, 0.97, 0.05),
            (1, 0, 0.012, 0.09, 0.02),
            (0, 2, 0.03, 0.2, 0.0, 1.0, 0.0, 0.0, 0.0, 0),
        ],
        loads=[(1, 0.9, 0.3), (2, 0.5, 0.2)], pvs=[(2, 0.6, 1.02)], slack=(0, 1.01, 0.05),
        shunts=[(1, 0.001, 0.15)])


def two_bus():
    return gridgen.PowerSystem.build(2, branches=[(0, 1, 0.0, 0.1, 0.0)], loads=[(1, 0.5, 0.2)],
                                     slack=(0, 1.0, 0.0))


def star_grid(n_leaf=1500, seed=3):
    """One hub bus joined to every other bus (hub degree > any tile), with a
    group of 5 parallel branches, a few chords and an isolated bus."""
    rng = np.random.default_rng(seed)
    n = n_leaf + 2                      # last bus isolated
    br = []
    for k in range(1, n_leaf + 1):
        br.append((0 if k % 2 else k, k if k % 2 else 0, rng.uniform(0.002, 0.02), rng.uniform(0.02, 0.2),
                   rng.uniform(0, 0.05), rng.choice([1.0, rng.uniform(0.95, 1.05)]),
                   rng.choice([0.0, 0.0, 0.0, rng.uniform(-0.1, 0.1)])))
    for _ in range(4):
        br.append((7, 0, 0.01, 0.05, 0.01))
    for _ in range(20):
        a, b = rng.choice(np.arange(1, n_leaf + 1), 2, replace=False)
        br.append((int(a), int(b), 0.01, 0.1, 0.0))
    loads = [(int(b), rng.uniform(0.01, 0.05), rng.uniform(0.0, 0.02)) for b in range(1, n)]
    pvs = [(int(b), 0.1, 1.01) for b in range(5, n_leaf, 50)]
    return gridgen.PowerSystem.build(n, branches=br, loads=loads, pvs=pvs, slack=(3, 1.0, 0.0),
                                     shunts=[(0, 0.0, 0.2), (9, 0.01, 0.1), (0, 0.0, 0.05)])


def edge_grid(seed=11):
    """Synthetic grid with end conductances, phase shifters, out-of-service
    branches and dense parallel groups."""
    s = gridgen.synthetic_grid(300, seed, n_branch=420, end_g_frac=0.3, xfmr_frac=0.3, shift_frac=0.5,
                               parallel_frac=0.05, cluster=30)
    s.br_status[::17] = 0
    return s


def state(sys, k, extended=False):
    return gridgen.flat_state(sys, extended) if k == 0 else gridgen.perturbed_state(sys, k, extended)


def with_outage(sys, l):
    s = sys.copy()
    if l >= 0:
        s.br_status = s.br_status.copy()
        s.br_status[l] = 0
    return s


def oracle_fj(sys, x, mode, **kw):
    F = oracle.residual(sys, x, mode, **kw)
    rp, ci, jv = oracle.jacobian(sys, x, mode) if not kw else oracle_jac_params(sys, x, mode, **kw)
    return F, rp, ci, jv


def oracle_jac_params(sys, x, mode, **kw):
    """Oracle Jacobian with branch parameters replaced (r, reac, b_c, tap)."""
    s = sys.copy()
    for k, name in (("r", "br_r"), ("reac", "br_x"), ("b_c", "br_b"), ("tap", "br_tap")):
        if kw.get(k) is not None:
            setattr(s, name, np.asarray(kw[k], float))
    return oracle.jacobian(s, x, mode)
