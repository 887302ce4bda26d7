"""The seeded generator's options (no GPU): the default grids do not depend on them, and each
option does what it states."""
import numpy as np
import pytest

import gridgen


def _connected(n, f, t):
    parent = np.arange(n)

    def root(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for a, b in zip(f, t):
        ra, rb = root(a), root(b)
        if ra != rb:
            parent[ra] = rb
    return len({root(a) for a in range(n)}) == 1


def test_defaults_unchanged_by_options():
    a = gridgen.synthetic_grid(3000, 11)
    b = gridgen.synthetic_grid(3000, 11, backbone="ring", pv_total=None, z_scale=1.0)
    for name in ("br_from", "br_to", "br_r", "br_x", "br_b", "br_tap", "pv_p", "load_p", "sh_b"):
        assert np.array_equal(getattr(a, name), getattr(b, name)), name


@pytest.mark.parametrize("backbone", ["ring", "mesh"])
def test_backbone_connected_and_sized(backbone):
    g = gridgen.synthetic_grid(5000, 3, backbone=backbone)
    assert g.n_branch == int(round(1.257 * 5000))
    assert _connected(g.n_bus, g.br_from, g.br_to)
    assert not np.any(g.br_from == g.br_to)


def test_mesh_ties_neighbouring_clusters_only():
    # clusters of 50 consecutive buses on a rectangle of ceil(sqrt(100)) = 10 columns
    g = gridgen.synthetic_grid(5000, 4, backbone="mesh", parallel_frac=0.0)
    cf, ct = g.br_from // 50, g.br_to // 50
    tie = cf != ct
    a, b = np.minimum(cf[tie], ct[tie]), np.maximum(cf[tie], ct[tie])
    right = (b == a + 1) & (a % 10 != 9)
    down = b == a + 10
    assert np.all(right | down)
    assert np.unique(a[right]).shape[0] == 90 and np.unique(a[down]).shape[0] == 90


def test_pv_total_and_z_scale():
    g = gridgen.synthetic_grid(2000, 5, pv_total=1.0, z_scale=0.25)
    assert np.isclose(g.pv_p.sum(), g.load_p.sum(), rtol=1e-12)
    h = gridgen.synthetic_grid(2000, 5)
    assert np.allclose(g.br_r, 0.25 * h.br_r, rtol=1e-15) and np.allclose(g.br_x, 0.25 * h.br_x, rtol=1e-15)
    assert np.array_equal(g.br_from, h.br_from) and np.array_equal(g.br_b, h.br_b)


def test_with_injections_sets_the_net_injections():
    import oracle
    g = gridgen.synthetic_grid(1500, 21)
    rng = np.random.default_rng(5)
    p, q, v = rng.normal(size=g.n_bus), rng.normal(size=g.n_bus), 1 + 0.01 * rng.normal(size=g.n_bus)
    h = gridgen.with_injections(g, p, q, v)
    p1, q1 = oracle.net_injections(h)
    is_pv = np.zeros(g.n_bus, bool)
    is_pv[g.pv_bus] = True
    assert np.array_equal(p1, p)
    assert np.array_equal(q1[~is_pv], q[~is_pv]) and not np.any(q1[is_pv])
    assert np.array_equal(h.pv_vset, v[g.pv_bus]) and h.slack_vset == v[g.slack_bus]
    for name in ("br_from", "br_to", "br_r", "br_x", "br_b", "br_tap", "br_shift", "sh_b"):
        assert np.array_equal(getattr(h, name), getattr(g, name)), name


def test_constructed_case_solved_from_flat_start():
    """A case built around target_state (injections = the network's own flows there) has that
    point as its solution, and flat-start Newton (the oracle's dense form) reaches it."""
    import oracle
    g = gridgen.synthetic_grid(300, 31)
    th, V = gridgen.target_state(g, 9)
    assert th[g.slack_bus] == g.slack_theta and np.all(np.abs(V - 1) <= 0.005)
    z = np.zeros(g.n_bus)
    fp, fq = oracle.bus_mismatch(g, th, V, p_inj=z, q_inj=z)
    h = gridgen.with_injections(g, fp, fq, V)
    xs = np.concatenate([th, V])
    assert np.max(np.abs(oracle.residual(h, xs))) == 0.0
    x, hist = oracle.newton_dense(h, gridgen.flat_state(h), tol=1e-10)
    assert hist[-1] <= 1e-10 and len(hist) <= 8
    np.testing.assert_allclose(x, xs, rtol=0, atol=1e-9)
