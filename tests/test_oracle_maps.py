"""Canonical index maps of the oracle (incidence list, contribution list)
against brute-force pure-Python loops over their definitions."""
import numpy as np
import pytest

import gridgen
import oracle
from oracle import REDUCED, EXTENDED


def grids():
    yield gridgen.PowerSystem.build(
        4, branches=[(0, 1, 0.01, 0.1, 0), (1, 0, 0.01, 0.1, 0), (1, 2, 0.01, 0.1, 0), (3, 1, 0.02, 0.1, 0)],
        pvs=[(2, 0.3, 1.0)], slack=(1, 1.0, 0.0), shunts=[(0, 0.0, 0.1), (0, 0.0, 0.2), (3, 0.01, 0.0)])
    yield gridgen.synthetic_grid(40, 5, n_branch=55, cluster=10)
    yield gridgen.synthetic_grid(13, 8, n_branch=20, cluster=13)


def brute_incidence(s):
    ptr = [0]
    code, other = [], []
    for o in range(s.n_bus):
        ent = []
        for k in range(s.n_branch):
            if s.br_from[k] == o:
                ent.append((int(s.br_to[k]), k, 0))
            if s.br_to[k] == o:
                ent.append((int(s.br_from[k]), k, 1))
        ent.sort()
        for oth, k, end in ent:
            code.append(2 * k + end)
            other.append(oth)
        ptr.append(len(code))
    return np.array(ptr), np.array(code), np.array(other)


@pytest.mark.parametrize("gi", range(3))
def test_incidence_lists_bruteforce(gi):
    s = list(grids())[gi]
    p, c, o = oracle.incidence_lists(s)
    bp, bc, bo = brute_incidence(s)
    assert np.array_equal(p, bp) and np.array_equal(c, bc) and np.array_equal(o, bo)


@pytest.mark.parametrize("mode", [REDUCED, EXTENDED])
@pytest.mark.parametrize("gi", range(3))
def test_contribution_lists_bruteforce(gi, mode):
    """Sources of each nonzero, by the definition: for (row of bus o, column of
    bus j) the branch ends at o whose other end is j (all ends of o when
    j == o), then the shunts of o in V-diagonal entries; -1 for constants."""
    s = list(grids())[gi]
    fm = oracle.Formulation(s, mode)
    n = s.n_bus
    x0 = gridgen.flat_state(s, mode == EXTENDED)
    rp, ci, _ = oracle.jacobian(s, x0, mode)
    ip, _, other = brute_incidence(s)
    cp, src = oracle.contribution_lists(s, mode)
    assert cp[-1] == src.shape[0] and cp.shape[0] == ci.shape[0] + 1
    for r in range(fm.n_rows):
        for k in range(rp[r], rp[r + 1]):
            c = ci[k]
            got = list(src[cp[k]:cp[k + 1]])
            ob = [b for b in range(n) if fm.row_p[b] == r or fm.row_q[b] == r]
            jb = [b for b in range(n) if fm.col_th[b] == c or fm.col_v[b] == c]
            if not ob or not jb:
                assert got == [-1]
                continue
            o, j = ob[0], jb[0]
            if j == o:
                want = list(range(ip[o], ip[o + 1]))
                if fm.col_v[o] == c:
                    want += [2 * s.n_branch + h for h in range(len(s.sh_bus)) if s.sh_bus[h] == o]
            else:
                want = [e for e in range(ip[o], ip[o + 1]) if other[e] == j]
            assert got == want, (r, c, got, want)
