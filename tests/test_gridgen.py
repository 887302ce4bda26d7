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
