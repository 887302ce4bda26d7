"""Seeded synthetic power-system inputs.

This module only draws inputs: network topology, branch and injection
parameters, operating states, branch outages, injection scalings and
cotangent vectors.  It contains none of the power-flow arithmetic (no
flows, no mismatches, no derivatives, no formulation index maps), so the
CPU oracle and the CUDA path can both consume its output without sharing
any of the method.

The test system of the paper (Sec. IV-A) is the Synthetic 70,000-bus grid
with 88,207 branches and transformers; that dataset is not available here.
``synthetic_grid`` builds a seeded stand-in with the same shape: clusters of
about 50 consecutive buses, each closed into a ring and meshed with random
chords, neighbouring clusters tied by 2-3 branches, about 1% parallel
branches, M/N = 1.257, 10% PV buses, 71.4% of buses carrying a PQ load and
4.3% carrying a shunt capacitor.  The branch model is the pi line / two
winding transformer of Sec. II-A with the end conductances of Eq. (4).

Every array is generated with numpy's PCG64 generator, whose streams are
identical on x86-64 and aarch64.
"""
from __future__ import annotations

from dataclasses import dataclass, field, fields
import math

import numpy as np

__all__ = [
    "PowerSystem",
    "synthetic_grid",
    "grid_200",
    "grid_70k",
    "flat_state",
    "perturbed_state",
    "target_state",
    "with_injections",
    "state_size",
    "gaussian_cotangents",
    "contingency_batch",
    "mixed_batch",
    "Instance",
]


@dataclass
class PowerSystem:
    """Plain arrays describing one network (per-unit, radians).

    Branch ``k`` joins ``br_from[k]`` to ``br_to[k]``: series impedance
    ``br_r + j br_x``, total line charging ``br_b`` (half at each end),
    off-nominal tap ``br_tap`` and phase shift ``br_shift`` on the from side,
    end shunt conductances ``br_g_fr`` / ``br_g_to`` (g_{L,h}, g_{L,k} of
    Eq. (4)) and ``br_status`` (0 = out of service).
    """

    n_bus: int
    br_from: np.ndarray
    br_to: np.ndarray
    br_r: np.ndarray
    br_x: np.ndarray
    br_b: np.ndarray
    br_tap: np.ndarray
    br_shift: np.ndarray
    br_g_fr: np.ndarray
    br_g_to: np.ndarray
    br_status: np.ndarray
    load_bus: np.ndarray
    load_p: np.ndarray
    load_q: np.ndarray
    pv_bus: np.ndarray
    pv_p: np.ndarray
    pv_vset: np.ndarray
    slack_bus: int
    slack_vset: float = 1.0
    slack_theta: float = 0.0
    sh_bus: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    sh_g: np.ndarray = field(default_factory=lambda: np.zeros(0))
    sh_b: np.ndarray = field(default_factory=lambda: np.zeros(0))

    @property
    def n_branch(self) -> int:
        return int(self.br_from.shape[0])

    @property
    def n_pv(self) -> int:
        return int(self.pv_bus.shape[0])

    def copy(self) -> "PowerSystem":
        kw = {}
        for f in fields(self):
            v = getattr(self, f.name)
            kw[f.name] = v.copy() if isinstance(v, np.ndarray) else v
        return PowerSystem(**kw)

    @staticmethod
    def build(n_bus, branches, loads=(), pvs=(), slack=(0, 1.0, 0.0), shunts=()):
        """Small hand-written systems.

        ``branches``: tuples (from, to, r, x, b[, tap[, shift[, g_fr[, g_to[, status]]]]]);
        ``loads``: (bus, P, Q); ``pvs``: (bus, P, Vset); ``slack``: (bus, Vset, theta);
        ``shunts``: (bus, g, b).
        """
        defaults = (0, 0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1)
        rows = [tuple(br) + defaults[len(br):] for br in branches]
        cols = list(zip(*rows)) if rows else [[] for _ in defaults]

        def arr(c, dt):
            return np.asarray(c, dtype=dt).reshape(-1)

        loads = list(loads)
        pvs = list(pvs)
        shunts = list(shunts)
        return PowerSystem(
            n_bus=int(n_bus),
            br_from=arr(cols[0], np.int32), br_to=arr(cols[1], np.int32),
            br_r=arr(cols[2], np.float64), br_x=arr(cols[3], np.float64),
            br_b=arr(cols[4], np.float64), br_tap=arr(cols[5], np.float64),
            br_shift=arr(cols[6], np.float64), br_g_fr=arr(cols[7], np.float64),
            br_g_to=arr(cols[8], np.float64), br_status=arr(cols[9], np.uint8),
            load_bus=arr([l[0] for l in loads], np.int32),
            load_p=arr([l[1] for l in loads], np.float64),
            load_q=arr([l[2] for l in loads], np.float64),
            pv_bus=arr([g[0] for g in pvs], np.int32),
            pv_p=arr([g[1] for g in pvs], np.float64),
            pv_vset=arr([g[2] for g in pvs], np.float64),
            slack_bus=int(slack[0]), slack_vset=float(slack[1]), slack_theta=float(slack[2]),
            sh_bus=arr([s[0] for s in shunts], np.int32),
            sh_g=arr([s[1] for s in shunts], np.float64),
            sh_b=arr([s[2] for s in shunts], np.float64),
        )


# --------------------------------------------------------------------------
# topology
# --------------------------------------------------------------------------

def _ring_of_meshes(n_bus: int, n_branch: int, rng: np.random.Generator, cluster: int,
                    parallel_frac: float, backbone: str = "ring"):
    n_cl = max(1, int(round(n_bus / cluster)))
    bounds = np.linspace(0, n_bus, n_cl + 1).round().astype(np.int64)
    start, size = bounds[:-1], np.diff(bounds)

    # ring inside every cluster (a single edge for a 2-bus cluster)
    ring_f, ring_t = [], []
    big = size >= 3
    if big.any():
        s, c = start[big], size[big]
        base = np.repeat(s, c)
        off = np.arange(c.sum()) - np.repeat(np.cumsum(c) - c, c)
        ring_f.append(base + off)
        ring_t.append(base + (off + 1) % np.repeat(c, c))
    two = size == 2
    if two.any():
        ring_f.append(start[two])
        ring_t.append(start[two] + 1)
    f = np.concatenate(ring_f) if ring_f else np.zeros(0, np.int64)
    t = np.concatenate(ring_t) if ring_t else np.zeros(0, np.int64)

    # ties between neighbouring clusters: the clusters arranged in a ring, or
    # ("mesh") row by row on a rectangle, each tied to its right and lower
    # neighbour
    if n_cl > 1:
        if backbone == "ring":
            n_links = n_cl if n_cl > 2 else 1
            k = np.arange(n_links)
            nxt = (k + 1) % n_cl
        elif backbone == "mesh":
            cols = int(np.ceil(np.sqrt(n_cl)))
            c = np.arange(n_cl)
            right = c[(c % cols != cols - 1) & (c + 1 < n_cl)]
            down = c[c + cols < n_cl]
            k = np.concatenate([right, down])
            nxt = np.concatenate([right + 1, down + cols])
            n_links = k.shape[0]
        else:
            raise ValueError("backbone must be 'ring' or 'mesh'")
        n_tie = rng.integers(2, 4, size=n_links)
        ka, kb = np.repeat(k, n_tie), np.repeat(nxt, n_tie)
        ta = start[ka] + rng.integers(0, size[ka])
        tb = start[kb] + rng.integers(0, size[kb])
        f, t = np.concatenate([f, ta]), np.concatenate([t, tb])

    n_par = int(round(parallel_frac * n_branch))
    n_chord = n_branch - f.shape[0] - n_par
    if n_chord < 0:
        raise ValueError(f"n_branch={n_branch} too small for a ring-of-meshes on {n_bus} buses")
    if n_chord > 0:
        ok = np.flatnonzero(size >= 2)
        p = size[ok] / size[ok].sum()
        cl = ok[rng.choice(ok.shape[0], size=n_chord, p=p)]
        u = rng.integers(0, size[cl])
        v = (u + rng.integers(1, size[cl])) % size[cl]
        f = np.concatenate([f, start[cl] + u])
        t = np.concatenate([t, start[cl] + v])
    if n_par > 0:
        dup = rng.integers(0, f.shape[0], size=n_par)
        f, t = np.concatenate([f, f[dup]]), np.concatenate([t, t[dup]])

    # random orientation, then shuffle branch order so ids carry no structure
    flip = rng.random(f.shape[0]) < 0.5
    f, t = np.where(flip, t, f), np.where(flip, f, t)
    perm = rng.permutation(f.shape[0])
    return f[perm].astype(np.int32), t[perm].astype(np.int32)


def synthetic_grid(n_bus: int, seed: int, *, n_branch: int | None = None,
                   pv_frac: float = 0.10, load_frac: float = 0.714,
                   shunt_frac: float = 0.043, xfmr_frac: float = 0.12,
                   shift_frac: float = 0.01, end_g_frac: float = 0.0,
                   parallel_frac: float = 0.01, cluster: int = 50,
                   n_pv: int | None = None, n_load: int | None = None,
                   n_shunt: int | None = None, load_scale: float = 1.0,
                   backbone: str = "ring", pv_total: float | None = None,
                   z_scale: float = 1.0) -> PowerSystem:
    """Ring-of-meshes grid with the parameter distributions of the paper-shaped workloads.

    r ~ U[0.002, 0.02], x = r * U[5, 12], b ~ U[0, 0.05]; a fraction
    ``xfmr_frac`` of branches are transformers with tap ~ U[0.95, 1.05], and a
    fraction ``shift_frac`` of those also get a phase shift ~ U[-0.1, 0.1] rad.
    Loads: P ~ U[0.1, 1.0] * load_scale, power factor ~ U[0.9, 0.98].
    PV: P = 1.03 * sum(P_load) / (N_PV + 1) * U[0.5, 1.5], Vset ~ U[0.98, 1.05].
    Shunt capacitors: g = 0, b ~ U[0, 0.3].  Slack: V = 1, theta = 0.
    ``end_g_frac`` of branches get end conductances g_fr, g_to ~ U[0, 0.01].
    """
    if n_bus < 2:
        raise ValueError("need at least 2 buses")
    rng = np.random.default_rng(seed)
    if n_branch is None:
        n_branch = int(round(1.257 * n_bus))
    f, t = _ring_of_meshes(n_bus, n_branch, rng, cluster, parallel_frac, backbone)
    m = f.shape[0]

    r = rng.uniform(0.002, 0.02, m) * z_scale
    x = r * rng.uniform(5.0, 12.0, m)
    b = rng.uniform(0.0, 0.05, m)
    tap = np.ones(m)
    shift = np.zeros(m)
    is_x = rng.random(m) < xfmr_frac
    tap[is_x] = rng.uniform(0.95, 1.05, int(is_x.sum()))
    xi = np.flatnonzero(is_x)
    has_shift = xi[rng.random(xi.shape[0]) < shift_frac]
    shift[has_shift] = rng.uniform(-0.1, 0.1, has_shift.shape[0])
    g_fr = np.zeros(m)
    g_to = np.zeros(m)
    if end_g_frac > 0:
        eg = rng.random(m) < end_g_frac
        g_fr[eg] = rng.uniform(0.0, 0.01, int(eg.sum()))
        g_to[eg] = rng.uniform(0.0, 0.01, int(eg.sum()))

    slack = int(rng.integers(0, n_bus))
    others = np.delete(np.arange(n_bus), slack)
    n_pv = int(round(pv_frac * n_bus)) if n_pv is None else n_pv
    n_pv = min(n_pv, n_bus - 1)
    # PV units spread along the bus order: one per stratum of consecutive
    # buses, so every cluster ring carries generation every few buses
    edges = np.linspace(0, others.shape[0], n_pv + 1).round().astype(np.int64)
    pv_bus = others[edges[:-1] + (rng.random(n_pv) * np.diff(edges)).astype(np.int64)]
    pv_bus = np.sort(pv_bus).astype(np.int32)
    n_load = int(round(load_frac * n_bus)) if n_load is None else n_load
    load_bus = np.sort(rng.choice(n_bus, size=min(n_load, n_bus), replace=False)).astype(np.int32)
    load_p = rng.uniform(0.1, 1.0, load_bus.shape[0]) * load_scale
    pf = rng.uniform(0.9, 0.98, load_bus.shape[0])
    load_q = load_p * np.tan(np.arccos(pf))
    pv_p = 1.03 * load_p.sum() / (n_pv + 1) * rng.uniform(0.5, 1.5, n_pv)
    if pv_total is not None and n_pv > 0:
        # PV outputs rescaled so that they add up to pv_total times the load
        pv_p = pv_p * (pv_total * load_p.sum() / pv_p.sum())
    pv_vset = rng.uniform(0.98, 1.05, n_pv)
    n_shunt = int(round(shunt_frac * n_bus)) if n_shunt is None else n_shunt
    sh_bus = np.sort(rng.choice(n_bus, size=min(n_shunt, n_bus), replace=False)).astype(np.int32)
    sh_g = np.zeros(sh_bus.shape[0])
    sh_b = rng.uniform(0.0, 0.3, sh_bus.shape[0])

    return PowerSystem(
        n_bus=n_bus, br_from=f, br_to=t, br_r=r, br_x=x, br_b=b, br_tap=tap,
        br_shift=shift, br_g_fr=g_fr, br_g_to=g_to,
        br_status=np.ones(m, np.uint8),
        load_bus=load_bus, load_p=load_p, load_q=load_q,
        pv_bus=pv_bus, pv_p=pv_p, pv_vset=pv_vset,
        slack_bus=slack, slack_vset=1.0, slack_theta=0.0,
        sh_bus=sh_bus, sh_g=sh_g, sh_b=sh_b,
    )


def grid_200(seed: int = 200, **kw) -> PowerSystem:
    """200-bus case: ~250 branches, 40 PV, 150 PQ loads, 10 shunts, 10% transformers."""
    args = dict(n_branch=250, n_pv=40, n_load=150, n_shunt=10, xfmr_frac=0.10)
    args.update(kw)
    return synthetic_grid(200, seed, **args)


def grid_70k(seed: int = 70000, **kw) -> PowerSystem:
    """70,000-bus case: ~88,000 branches, 7,000 PV, 50,000 PQ loads, 3,000 shunts, 12% transformers."""
    args = dict(n_branch=88000, n_pv=7000, n_load=50000, n_shunt=3000, xfmr_frac=0.12)
    args.update(kw)
    return synthetic_grid(70000, seed, **args)


# --------------------------------------------------------------------------
# operating states, cotangents
# --------------------------------------------------------------------------

def state_size(sys: PowerSystem, extended: bool) -> int:
    """Length of the state vector: [theta(N), V(N)] plus [Q_g (PV gens, then slack), P_s]
    in the extended formulation (Eq. 3)."""
    n = 2 * sys.n_bus
    if extended:
        n += sys.n_pv + 2
    return n


def flat_state(sys: PowerSystem, extended: bool = False) -> np.ndarray:
    """theta = 0 (slack: its set angle), V = 1 (PV and slack buses: their set voltage)."""
    n = sys.n_bus
    x = np.zeros(state_size(sys, extended))
    x[n:2 * n] = 1.0
    x[n + sys.pv_bus] = sys.pv_vset
    x[n + sys.slack_bus] = sys.slack_vset
    x[sys.slack_bus] = sys.slack_theta
    return x


def perturbed_state(sys: PowerSystem, seed: int, extended: bool = False,
                    theta_max: float = 0.2, v_lo: float = 0.95, v_hi: float = 1.05) -> np.ndarray:
    """theta ~ U[-0.2, 0.2], V ~ U[0.95, 1.05]; Q_g, P_s ~ U[-1, 1] in the extended layout."""
    rng = np.random.default_rng(seed)
    n = sys.n_bus
    x = np.empty(state_size(sys, extended))
    x[:n] = rng.uniform(-theta_max, theta_max, n)
    x[n:2 * n] = rng.uniform(v_lo, v_hi, n)
    if extended:
        x[2 * n:] = rng.uniform(-1.0, 1.0, x.shape[0] - 2 * n)
    return x


def target_state(sys: PowerSystem, seed: int, theta_max: float = 0.003,
                 dv: float = 0.005) -> tuple[np.ndarray, np.ndarray]:
    """An operating point (theta, V) to build a solvable case around:
    theta ~ U[-theta_max, theta_max] (the slack at its set angle), V ~ 1 + U[-dv, dv].

    A case whose injections are the network's own flows at this point (see
    ``with_injections``) has it as a power-flow solution; the small spread
    keeps the flows, and the losses the slack must cover, small enough for
    flat-start Newton to reach it on the long ring of the 70k-bus grid."""
    rng = np.random.default_rng(seed)
    theta = rng.uniform(-theta_max, theta_max, sys.n_bus)
    theta[sys.slack_bus] = sys.slack_theta
    V = 1.0 + rng.uniform(-dv, dv, sys.n_bus)
    return theta, V


def with_injections(sys: PowerSystem, p_inj: np.ndarray, q_inj: np.ndarray,
                    v_set: np.ndarray) -> PowerSystem:
    """A copy of ``sys`` whose per-bus net injections are ``p_inj``, ``q_inj``
    (P_g - P_L, Q_g - Q_L) and whose PV units and slack hold the voltages
    ``v_set`` of their buses.

    Network unchanged; every PV unit produces the bus's p_inj; every other bus
    (the slack included) carries one load of -p_inj, -q_inj.  A PV bus's Q
    injection becomes 0 (its Q is a free variable of the power flow)."""
    n = sys.n_bus
    p_inj = np.asarray(p_inj, np.float64)
    q_inj = np.asarray(q_inj, np.float64)
    v_set = np.asarray(v_set, np.float64)
    if p_inj.shape != (n,) or q_inj.shape != (n,) or v_set.shape != (n,):
        raise ValueError("p_inj, q_inj and v_set need one value per bus")
    if np.unique(sys.pv_bus).shape[0] != sys.n_pv:
        raise ValueError("with_injections needs at most one PV unit per bus")
    out = sys.copy()
    is_pv = np.zeros(n, bool)
    is_pv[sys.pv_bus] = True
    load_bus = np.flatnonzero(~is_pv).astype(np.int32)
    out.load_bus = load_bus
    out.load_p = -p_inj[load_bus]
    out.load_q = -q_inj[load_bus]
    out.pv_p = p_inj[sys.pv_bus].copy()
    out.pv_vset = v_set[sys.pv_bus].copy()
    out.slack_vset = float(v_set[sys.slack_bus])
    return out


def gaussian_cotangents(n_rows: int, n_cot: int, seed: int = 4000) -> np.ndarray:
    """(n_cot, n_rows) standard normal cotangents; row k uses seed ``seed + k``."""
    out = np.empty((n_cot, n_rows))
    for k in range(n_cot):
        out[k] = np.random.default_rng(seed + k).standard_normal(n_rows)
    return out


# --------------------------------------------------------------------------
# batched workloads
# --------------------------------------------------------------------------

@dataclass
class Instance:
    """One evaluation instance of a batch: a grid, a state, optional branch
    outage and optional per-bus net-injection overrides (P_g - P_L, Q_g - Q_L)."""

    grid: int
    x: np.ndarray
    outage: int = -1
    p_inj: np.ndarray | None = None
    q_inj: np.ndarray | None = None


def contingency_batch(seed: int = 3000, n_small: int = 2048, n_large: int = 256,
                      small_bus: int = 2000, large_bus: int = 10000, only=None):
    """2,048 instances of a 2,000-bus grid plus 256 of a 10,000-bus grid; each
    instance has its own seeded perturbed state and one seeded branch outage.
    only: indices of the instances to generate (the others are left out of the
    returned list; each generated one equals its entry in the full batch)."""
    grids = [synthetic_grid(small_bus, seed), synthetic_grid(large_bus, seed + 1)]
    rng = np.random.default_rng(seed + 2)
    keep = None if only is None else set(int(i) for i in only)
    insts = []
    j = 0
    for gi, count in ((0, n_small), (1, n_large)):
        g = grids[gi]
        outs = rng.integers(0, g.n_branch, size=count)
        for k in range(count):
            if keep is None or j in keep:
                insts.append(Instance(grid=gi, x=perturbed_state(g, seed * 7919 + 1000003 * gi + k),
                                      outage=int(outs[k])))
            j += 1
    return grids, insts


def mixed_batch(n_inst: int = 4096, seed: int = 5000, n_min: int = 500, n_max: int = 20000, only=None):
    """Mixed-scenario batch: every instance has its own grid with a log-uniform
    size in [n_min, n_max]; PV outputs scaled per generator by U[0.5, 1.5] and
    loads by one U[0.8, 1.2] factor per instance, given as net-injection
    overrides.  only: indices of the instances to generate (grid k of a
    generated instance k is the full batch's grid k; `grid` then indexes the
    returned list)."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(math.log(n_min), math.log(n_max), n_inst)).round().astype(int)
    keep = None if only is None else set(int(i) for i in only)
    grids, insts = [], []
    for k, n in enumerate(sizes):
        if keep is not None and k not in keep:
            continue
        g = synthetic_grid(int(n), seed + 17 * k + 1)
        r = np.random.default_rng(seed * 31 + k)
        pv_scale = r.uniform(0.5, 1.5, g.n_pv)
        load_scale = r.uniform(0.8, 1.2)
        p = np.zeros(g.n_bus)
        q = np.zeros(g.n_bus)
        np.add.at(p, g.pv_bus, g.pv_p * pv_scale)
        np.add.at(p, g.load_bus, -g.load_p * load_scale)
        np.add.at(q, g.load_bus, -g.load_q * load_scale)
        grids.append(g)
        insts.append(Instance(grid=len(grids) - 1, x=perturbed_state(g, seed * 131 + k), p_inj=p, q_inj=q))
    return grids, insts
