"""CUDA path vs the CPU oracle through the C ABI: bit-exact index maps, F and
J values within 1e-12 rel / 1e-10 abs, determinism across runs and tunings,
edge cases.  GPU only."""
import numpy as np
import pytest
import torch

import gridgen
import oracle
from oracle import REDUCED, EXTENDED
from tests.gpu_common import assert_tol, edge_grid, star_grid, state, three_bus, two_bus

pytestmark = pytest.mark.gpu

MODES = [REDUCED, EXTENDED]
MNAME = {REDUCED: "reduced", EXTENDED: "extended"}


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2011_11880_gb300 as p
    return p


def grids():
    return {
        "two_bus": two_bus(),
        "three_bus": three_bus(),
        "grid30": gridgen.synthetic_grid(30, 7, n_branch=39, end_g_frac=0.2, xfmr_frac=0.3, shift_frac=0.3,
                                         cluster=10),
        "grid200": gridgen.grid_200(),
        "edge300": edge_grid(),
        "star": star_grid(),
        "grid2000": gridgen.synthetic_grid(2000, 21),
    }


GRIDS = grids()


def gpu_eval(P, sys, x_np, mode, tuning=None):
    ctx = P.Context(sys, MNAME[mode])
    if tuning:
        ctx.set_tuning(*tuning)
    x = torch.from_numpy(x_np).cuda()
    F, v = ctx.residual_jacobian(x)
    torch.cuda.synchronize()
    return ctx, F.cpu().numpy(), v.cpu().numpy()


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("name", list(GRIDS))
def test_pattern_and_maps_bit_exact(P, name, mode):
    sys = GRIDS[name]
    ctx = P.Context(sys, MNAME[mode])
    rp, ci = ctx.pattern()
    x0 = gridgen.flat_state(sys, mode == EXTENDED)
    rpo, cio, _ = oracle.jacobian(sys, x0, mode)
    assert np.array_equal(rp, rpo) and np.array_equal(ci, cio)
    ip, code, oth = ctx.incidence()
    ipo, codeo, otho = oracle.incidence_lists(sys)
    assert np.array_equal(ip, ipo) and np.array_equal(code, codeo) and np.array_equal(oth, otho)
    if sys.n_bus <= 2000:
        cp, src = ctx.contributions()
        cpo, srco = oracle.contribution_lists(sys, mode)
        assert np.array_equal(cp, cpo) and np.array_equal(src, srco)
    d = ctx.dims
    fm = oracle.Formulation(sys, mode)
    assert d.n_f == fm.n_rows and d.nnz == rpo[-1] and d.n_x == x0.shape[0]
    ctx.check_device()


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("name", list(GRIDS))
def test_values_match_oracle(P, name, mode):
    sys = GRIDS[name]
    for k in (0, 1, 2):
        x = state(sys, k, mode == EXTENDED)
        ctx, F, v = gpu_eval(P, sys, x, mode)
        assert_tol(F, oracle.residual(sys, x, mode), f"{name} F state {k}")
        assert_tol(v, oracle.jacobian(sys, x, mode)[2], f"{name} J state {k}")
        ctx.check_device()


@pytest.mark.parametrize("mode", MODES)
def test_200bus_six_states_split_and_fused(P, mode):
    """Config 1: flat start and 5 perturbed states; F only, J only and fused agree bit for bit."""
    sys = gridgen.grid_200()
    ctx = P.Context(sys, MNAME[mode])
    for k in range(6):
        xn = state(sys, k, mode == EXTENDED)
        x = torch.from_numpy(xn).cuda()
        F1 = ctx.residual(x)
        v1 = ctx.jacobian(x)
        F2, v2 = ctx.residual_jacobian(x)
        assert torch.equal(F1, F2) and torch.equal(v1, v2)
        assert_tol(F1.cpu().numpy(), oracle.residual(sys, xn, mode), f"F {k}")
        assert_tol(v1.cpu().numpy(), oracle.jacobian(sys, xn, mode)[2], f"J {k}")


def test_zero_residual_at_oracle_solution(P):
    """F at the oracle's Newton solution of the 200-bus case is <= 1e-10."""
    sys = gridgen.grid_200()
    xs, hist = oracle.newton_dense(sys, gridgen.flat_state(sys))
    assert hist[-1] <= 1e-10
    ctx = P.Context(sys)
    F = ctx.residual(torch.from_numpy(xs).cuda()).cpu().numpy()
    assert np.max(np.abs(F)) <= 1e-10


@pytest.mark.parametrize("name", ["grid200", "star", "edge300"])
def test_deterministic_across_runs_and_tunings(P, name):
    sys = GRIDS[name]
    x = torch.from_numpy(state(sys, 3)).cuda()
    ctx = P.Context(sys)
    F0, v0 = ctx.residual_jacobian(x)
    for _ in range(3):
        F1, v1 = ctx.residual_jacobian(x)
        assert torch.equal(F0, F1) and torch.equal(v0, v1)
    nan = float("nan")
    for fuse in (0, 1):
        for split in (0, 1, 2):
            for tile in (32, 64, 96, 128):
                for ctas in (0, 1, 3, 16):
                    ctx.set_tuning(tile, ctas, split, fuse)
                    for _ in range(2):                     # a persistent grid's counters are reused
                        F1, v1 = ctx.residual_jacobian(x, ctx.empty_f().fill_(nan), ctx.empty_vals().fill_(nan))
                        assert torch.equal(F0, F1) and torch.equal(v0, v1), (tile, ctas, split, fuse)
                    F2 = ctx.residual(x, ctx.empty_f().fill_(nan))   # F alone takes the same sums
                    assert torch.equal(F0, F2), (tile, ctas, split, fuse)
                    ctx.check_device()


def test_autotune_keeps_results(P):
    sys = gridgen.synthetic_grid(2000, 5)
    ctx = P.Context(sys)
    x = torch.from_numpy(state(sys, 2)).cuda()
    F0, v0 = ctx.residual_jacobian(x)
    F, v = torch.empty_like(F0), torch.empty_like(v0)
    t = ctx.autotune(x, F, v)
    assert t["tile_inc"] in (32, 64, 96, 128)
    F1, v1 = ctx.residual_jacobian(x)
    assert torch.equal(F0, F1) and torch.equal(v0, v1)


def test_host_entry_point_matches_device(P):
    sys = GRIDS["edge300"]
    ctx = P.Context(sys)
    xn = state(sys, 4)
    F_d, v_d = ctx.residual_jacobian(torch.from_numpy(xn).cuda())
    F_h = np.empty(ctx.dims.n_f)
    v_h = np.empty(ctx.dims.nnz)
    ctx.residual_jacobian_host(xn, F_h, v_h)
    assert np.array_equal(F_h, F_d.cpu().numpy()) and np.array_equal(v_h, v_d.cpu().numpy())


def test_parameter_overrides_match_oracle(P):
    """pf_eval with per-call r, x, b_c, tap and injection overrides."""
    sys = GRIDS["grid30"]
    rng = np.random.default_rng(0)
    r = sys.br_r * rng.uniform(0.8, 1.2, sys.n_branch)
    xr = sys.br_x * rng.uniform(0.8, 1.2, sys.n_branch)
    b = sys.br_b * rng.uniform(0.5, 1.5, sys.n_branch)
    tap = sys.br_tap * rng.uniform(0.98, 1.02, sys.n_branch)
    p0, q0 = oracle.net_injections(sys)
    p = p0 + rng.normal(0, 0.1, sys.n_bus)
    q = q0 + rng.normal(0, 0.1, sys.n_bus)
    xn = state(sys, 2)
    ctx = P.Context(sys)
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    F, v = ctx.eval(c(xn), ctx.empty_f(), ctx.empty_vals(), br_r=c(r), br_x=c(xr), br_b=c(b), br_tap=c(tap),
                    p_inj=c(p), q_inj=c(q))
    s2 = sys.copy()
    s2.br_r, s2.br_x, s2.br_b, s2.br_tap = r, xr, b, tap
    assert_tol(F.cpu().numpy(), oracle.residual(s2, xn, REDUCED, p_inj=p, q_inj=q), "F overrides")
    assert_tol(v.cpu().numpy(), oracle.jacobian(s2, xn, REDUCED)[2], "J overrides")
    # without overrides the built values come back
    F0 = ctx.residual(c(xn)).cpu().numpy()
    assert_tol(F0, oracle.residual(sys, xn), "F built")


def test_full_70k_against_oracle(P):
    """Config 2: the 70,000-bus grid, every F row and J value, 3 of the 10 states."""
    sys = gridgen.grid_70k()
    ctx = P.Context(sys)
    rp, ci = ctx.pattern()
    rpo, cio, _ = oracle.jacobian(sys, gridgen.flat_state(sys))
    assert np.array_equal(rp, rpo) and np.array_equal(ci, cio)
    for k in (0, 1, 10):
        xn = state(sys, k)
        F, v = ctx.residual_jacobian(torch.from_numpy(xn).cuda())
        assert_tol(F.cpu().numpy(), oracle.residual(sys, xn), f"70k F {k}")
        assert_tol(v.cpu().numpy(), oracle.jacobian(sys, xn)[2], f"70k J {k}")
    ctx.check_device()


def test_full_70k_extended_against_oracle(P):
    """The 70,000-bus grid in the paper's extended formulation (Sec. II-A, Eqs. 1-3): the pattern
    bit-exact, every F row and J value at the flat start and two perturbed states."""
    sys = gridgen.grid_70k()
    ctx = P.Context(sys, "extended")
    rp, ci = ctx.pattern()
    rpo, cio, _ = oracle.jacobian(sys, gridgen.flat_state(sys, True), EXTENDED)
    assert np.array_equal(rp, rpo) and np.array_equal(ci, cio)
    for k in (0, 1, 10):
        xn = state(sys, k, extended=True)
        F, v = ctx.residual_jacobian(torch.from_numpy(xn).cuda())
        assert_tol(F.cpu().numpy(), oracle.residual(sys, xn, EXTENDED), f"70k extended F {k}")
        assert_tol(v.cpu().numpy(), oracle.jacobian(sys, xn, EXTENDED)[2], f"70k extended J {k}")
    ctx.check_device()


def test_phasor_routine_against_libm(P):
    """The table-driven sin / cos of the phasor kernel vs the host libm (numpy): the fixed-point
    path (|t| < 32) on a grid, at and between table points, near the switch to sincos() at 32, on
    tiny and subnormal angles; and arguments past it."""
    ctx = P.Context(GRIDS["three_bus"])
    rng = np.random.default_rng(0)
    steps = np.arange(-3000, 3001) * (np.pi / 16384)           # table points and the midpoints between
    th = np.concatenate([np.linspace(-7, 7, 400001), rng.uniform(-1e4, 1e4, 100000),
                         rng.uniform(-32, 32, 100000), steps, steps + np.pi / 32768,
                         np.nextafter(32.0, 0.0) * np.array([1.0, -1.0]), [32.0, -32.0],
                         2.0 ** -np.arange(1, 1075, 7.0), -(2.0 ** -np.arange(1, 1075, 11.0)), [5e-324],
                         [0.0, -0.0, np.pi, -np.pi, 1e5, -3e6, 65535.9, 65536.0]])
    c, s = ctx.sincos(torch.from_numpy(th).cuda())
    c, s = c.cpu().numpy(), s.cpu().numpy()
    small = np.abs(th) <= 32
    # sin is odd: the sign of a tiny or zero angle is kept
    tiny = np.abs(th) < 1e-300
    assert np.array_equal(np.signbit(s[tiny]), np.signbit(th[tiny]))
    assert np.max(np.abs(c - np.cos(th))[small]) <= 4.5e-16
    assert np.max(np.abs(s - np.sin(th))[small]) <= 4.5e-16
    # larger arguments: the reduction error grows with |theta| (ulp of theta)
    assert np.max(np.abs(c - np.cos(th))) <= 1e-12
    assert np.max(np.abs(s - np.sin(th))) <= 1e-12


def test_voltage_records_against_libm(P):
    """The per-bus records (V cos theta, V sin theta, V, 1/V) vs numpy, over a wide range of V,
    and the dead-bus substitution (|V| < 2^-500: 2^-600 in place of V)."""
    sys = GRIDS["grid2000"]
    ctx = P.Context(sys)
    n = sys.n_bus
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.uniform(-7, 7, n), np.exp(rng.uniform(-40, 40, n))])
    x[n + 1::7] *= -1.0                                      # negative magnitudes too
    x[n + 3], x[n + 4], x[n + 5] = 0.0, 1e-200, 2.0 ** -499
    rec = ctx.voltage_records(torch.from_numpy(x).cuda()).cpu().numpy()
    th, vm = x[:n], x[n:]
    dead = np.abs(vm) < 2.0 ** -500
    assert dead.sum() == 2 and np.array_equal(rec[:, 2], vm)
    sv = np.where(dead, 2.0 ** -600, vm)
    # products of the phasor routine (|error| <= 4.5e-16) and V, rounded once
    assert np.all(np.abs(rec[:, 0] - sv * np.cos(th)) <= 8e-16 * np.abs(sv))
    assert np.all(np.abs(rec[:, 1] - sv * np.sin(th)) <= 8e-16 * np.abs(sv))
    # 1/V within one ulp
    r = 1.0 / sv
    assert np.all(np.abs(rec[:, 3] - r) <= np.spacing(np.abs(r)))
    assert np.array_equal(rec[dead, 3], np.full(2, 2.0 ** 600))


@pytest.mark.parametrize("mode", MODES)
def test_dead_bus_matches_oracle(P, mode):
    """A PQ bus at V = 0 (and one at 1e-300): F and J (whose dF/dV values divide that factor
    out again) still match the oracle."""
    sys = GRIDS["grid200"]
    n = sys.n_bus
    x = state(sys, 2, mode == EXTENDED).copy()
    pq = [b for b in range(n) if b not in set(sys.pv_bus.tolist()) | {sys.slack_bus}]
    x[n + pq[3]] = 0.0
    x[n + pq[10]] = 1e-300
    ctx, F, v = gpu_eval(P, sys, x, mode)
    assert_tol(F, oracle.residual(sys, x, mode), "F dead bus")
    assert_tol(v, oracle.jacobian(sys, x, mode)[2], "J dead bus")


@pytest.mark.parametrize("mode", MODES)
def test_out_of_range_terms_match_oracle(P, mode):
    """Two connected buses at V = 1e10 make the pair terms X, Y about 1e20, beyond the exact
    integer bus sums' range (2^57): those buses sum in FP64; F and J still match the oracle."""
    sys = GRIDS["grid200"]
    n = sys.n_bus
    x = state(sys, 3, mode == EXTENDED).copy()
    a, b = int(sys.br_from[0]), int(sys.br_to[0])
    x[n + a] = 1e10
    x[n + b] = -2e10
    ctx, F, v = gpu_eval(P, sys, x, mode)
    assert np.max(np.abs(F)) > 2.0 ** 57
    assert_tol(F, oracle.residual(sys, x, mode), "F out of range")
    assert_tol(v, oracle.jacobian(sys, x, mode)[2], "J out of range")


@pytest.mark.parametrize("mode", MODES)
def test_split_rounds_bit_identical_under_masks(P, mode):
    """Smaller tiles (split rounds) and the records formed in the fused kernel give the
    default results bit for bit: a batch with outage instances, a per-call status mask,
    and (extended) generators held at limits."""
    grids = [GRIDS["grid200"], GRIDS["grid30"], GRIDS["edge300"]]
    inst = [(0, -1), (0, 7), (1, 3), (2, -1), (2, 11), (1, -1)]
    ctx = P.Context(grids, MNAME[mode], instances=inst)
    x = torch.from_numpy(np.concatenate([state(grids[g], k + 1, mode == EXTENDED)
                                         for k, (g, _) in enumerate(inst)])).cuda()
    rng = np.random.default_rng(8)
    status = torch.from_numpy((rng.random(ctx.dims.n_branch_inst) > 0.05).astype(np.uint8)).cuda()
    kw = {"status": status}
    if mode == EXTENDED:
        kw["gen_mode"] = torch.from_numpy(rng.integers(0, 3, ctx.dims.n_gen_inst).astype(np.uint8)).cuda()
        kw["gen_qlim"] = torch.from_numpy(rng.uniform(-0.5, 0.8, ctx.dims.n_gen_inst)).cuda()
    outs = []
    for fuse in (0, 1):
        for split in (0, 1, 2):
            for tile in (32, 128):
                ctx.set_tuning(tile, 0, split, fuse)
                outs.append(ctx.eval(x, ctx.empty_f(), ctx.empty_vals(), **kw))
                outs.append(ctx.residual_jacobian(x))
    for k in range(2, len(outs), 2):
        assert torch.equal(outs[0][0], outs[k][0]) and torch.equal(outs[0][1], outs[k][1]), k
        assert torch.equal(outs[1][0], outs[k + 1][0]) and torch.equal(outs[1][1], outs[k + 1][1]), k
    ctx.check_device()


@pytest.mark.parametrize("mode", MODES)
def test_persistent_schedule_bit_identical(P, mode):
    """Persistent fused grids (ctas_per_sm > 0), whose warps claim rounds from a counter, give
    the one-CTA-per-round results bit for bit over a batch: outage instances, a status mask,
    branch-parameter overrides, buses with more than 32 neighbours (the warp-per-bus kernel),
    F or J alone, repeated launches (the counters are reset by each grid), the fused stage
    launched alone, and replays of a captured CUDA graph."""
    grids = [GRIDS["grid200"], GRIDS["star"], GRIDS["edge300"]]
    inst = [(0, -1), (1, -1), (0, 7), (2, -1), (1, 5), (2, 11), (0, 3)]
    ctx = P.Context(grids, MNAME[mode], instances=inst)
    d = ctx.dims
    x = torch.from_numpy(np.concatenate([state(grids[g], k + 2, mode == EXTENDED)
                                         for k, (g, _) in enumerate(inst)])).cuda()
    rng = np.random.default_rng(21)
    r0 = np.concatenate([g.br_r for g in grids])
    assert r0.size == d.n_branch
    kw = {"status": torch.from_numpy((rng.random(d.n_branch_inst) > 0.05).astype(np.uint8)).cuda(),
          "br_r": torch.from_numpy(r0 * rng.uniform(0.9, 1.1, r0.size)).cuda()}
    if mode == EXTENDED:
        kw["gen_mode"] = torch.from_numpy(rng.integers(0, 3, d.n_gen_inst).astype(np.uint8)).cuda()
        kw["gen_qlim"] = torch.from_numpy(rng.uniform(-0.5, 0.8, d.n_gen_inst)).cuda()
    nan = float("nan")

    def run():   # outputs start as NaN, so a round left out cannot pass for a written one
        F, V = ctx.empty_f().fill_(nan), ctx.empty_vals().fill_(nan)
        ctx.eval_stage(1, x, F, V)
        ctx.eval_stage(2, x, F, V)
        # the fused stage alone right after the kernels that write the per-call coefficients
        Fo, Vo = ctx.empty_f().fill_(nan), ctx.empty_vals().fill_(nan)
        ctx.eval_stage(1, x, Fo, Vo, **kw)
        ctx.eval_stage(2, x, Fo, Vo, **kw)
        return (ctx.eval(x, ctx.empty_f().fill_(nan), ctx.empty_vals().fill_(nan), **kw),
                ctx.residual_jacobian(x, ctx.empty_f().fill_(nan), ctx.empty_vals().fill_(nan)),
                ctx.residual(x, ctx.empty_f().fill_(nan)), ctx.jacobian(x, ctx.empty_vals().fill_(nan)),
                (F, V), (Fo, Vo))

    ctx.set_tuning(64, 0, 0)
    ref = run()
    assert torch.equal(ref[5][0], ref[0][0]) and torch.equal(ref[5][1], ref[0][1])   # stages == one call
    assert torch.equal(ref[4][0], ref[1][0]) and torch.equal(ref[4][1], ref[1][1])
    for tile, cps, split, fuse in ((64, 16, 0, 0), (64, 20, 0, 0), (32, 1, 0, 0), (128, 16, 1, 0), (96, 3, 1, 0),
                                   (64, 0, 0, 1), (32, 4, 2, 1)):
        ctx.set_tuning(tile, cps, split, fuse)
        for _ in range(2):
            got = run()
            for k in (0, 1, 4, 5):
                assert torch.equal(ref[k][0], got[k][0]) and torch.equal(ref[k][1], got[k][1]), (k, tile, cps)
            assert torch.equal(ref[2], got[2]) and torch.equal(ref[3], got[3]), (tile, cps)
        ctx.check_device()                     # the schedule counters are back at zero
    s = torch.cuda.Stream()
    F, V = ctx.empty_f(), ctx.empty_vals()
    ctx.set_tuning(64, 16, 0)
    with torch.cuda.stream(s):
        ctx.residual_jacobian(x, F, V, stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ctx.residual_jacobian(x, F, V, stream=s)
    for _ in range(3):
        F.fill_(nan)
        V.fill_(nan)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(F, ref[1][0]) and torch.equal(V, ref[1][1])
    ctx.check_device()


def test_autotune_cache(P, tmp_path):
    """pf_autotune_cache: the first context times and appends its choice; a second context of
    the same shape takes it from the file without timing; another instance list is another key;
    lines that do not parse or hold out-of-range values are ignored.  Results never change."""
    sys = gridgen.synthetic_grid(2000, 5)
    path = tmp_path / "tuning.txt"
    x1 = np.concatenate([state(sys, 1), state(sys, 2)])
    x = torch.from_numpy(x1).cuda()

    def ctx_of(inst):
        c = P.Context([sys], instances=inst)
        return c, c.empty_f(), c.empty_vals()

    c1, F1, V1 = ctx_of([(0, -1), (0, 3)])
    t1 = c1.autotune(x, F1, V1, cache=str(path))
    assert t1["from_cache"] is False
    lines = path.read_text().splitlines()
    assert len(lines) == 1 and lines[0].startswith("pf-tuning-v2 ") and len(lines[0].split()) == 6
    c2, F2, V2 = ctx_of([(0, -1), (0, 3)])
    t2 = c2.autotune(x, F2, V2, cache=str(path))
    assert t2["from_cache"] is True and {k: t2[k] for k in t1 if k != "from_cache"} == \
        {k: t1[k] for k in t1 if k != "from_cache"}
    assert c2.tuning() == {k: t1[k] for k in t1 if k != "from_cache"}
    assert len(path.read_text().splitlines()) == 1
    a1, b1 = c1.residual_jacobian(x)
    a2, b2 = c2.residual_jacobian(x)
    assert torch.equal(a1, a2) and torch.equal(b1, b2)
    c3, F3, V3 = ctx_of([(0, -1), (0, 4)])             # another outage: another key
    assert c3.autotune(x, F3, V3, cache=str(path))["from_cache"] is False
    assert len(path.read_text().splitlines()) == 2
    key = lines[0].split()[1]
    # an out-of-range tile, CTA count and phasor form, and a line of the older format
    path.write_text(f"garbage line\npf-tuning-v2 {key} 48 0 0 0\npf-tuning-v2 {key} 64 99 0 0\n"
                    f"pf-tuning-v2 {key} 64 0 0 2\npf-tuning-v1 {key} 64 0 0\n")
    c4, F4, V4 = ctx_of([(0, -1), (0, 3)])
    assert c4.autotune(x, F4, V4, cache=str(path))["from_cache"] is False   # nothing valid: timed again
    assert len(path.read_text().splitlines()) == 6
    c5, F5, V5 = ctx_of([(0, -1), (0, 3)])
    assert c5.autotune(x, F5, V5, cache=str(path))["from_cache"] is True
    for c in (c1, c2, c3, c4, c5):
        c.check_device()


@pytest.mark.parametrize("mode", MODES)
def test_wide_bus_sums_match_oracle(P, mode):
    """A hub with 16 branches of |y| ~ 1000 at V = 1.99 and equal angles: its exact bus sums
    exceed 64 bits at the kernel's fixed-point scale (16 terms of about 2^61), so the hub takes
    the FP64 form; F and J match the oracle, and every tuning gives the same bits."""
    from gridgen import PowerSystem
    n = 18
    br = [(0, k, 1e-5, 1e-3) for k in range(1, 17)] + [(16, 17, 0.01, 0.1)]
    sys = PowerSystem.build(n, br, loads=[(0, 0.5, 0.1)], pvs=[(5, 0.2, 1.99)], slack=(17, 1.99, 0.0))
    x = np.zeros(gridgen.state_size(sys, mode == EXTENDED))
    x[n:2 * n] = 1.99
    ctx, F, v = gpu_eval(P, sys, x, mode)
    # the hub's dF_P/dtheta_o is its sum S_Y itself (the flows cancel in F at equal voltages)
    assert np.max(np.abs(v)) > 5e4
    assert_tol(F, oracle.residual(sys, x, mode), "F wide sums")
    assert_tol(v, oracle.jacobian(sys, x, mode)[2], "J wide sums")
    for tile in (32, 96):
        _, F2, v2 = gpu_eval(P, sys, x, mode, (tile, 0, 0, 0))
        assert np.array_equal(F2, F) and np.array_equal(v2, v)
