"""Benchmark: F+J evaluations/s on the 70,000-bus synthetic grid (one GPU per rank).

One step = one batched launch that evaluates the bus mismatches F and the
Jacobian values J (tasks 1 and 2 of Newton power flow) at 48 Newton-like
states of the grid (48 instances of one context; k_phasor_fx + k_tile,
replayed as a captured CUDA graph) through the library's C ABI.  Inputs are
resident in HBM; the 48 states' x, F and J (444 MB) exceed the 129 MB L2.
value = evaluations / s.  The same states evaluated one launch at a time are
reported beside it ("single_instance"), on the same GPU.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun every rank evaluates its own replica (the path does not
shard); value = evaluations of all ranks / max rank time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gridgen  # noqa: E402

N_STATES = 48
LEAD_BYTES = 1 << 30
METRIC = "F+J evals/s on 70k-bus grid (batched; single-instance reported beside)"
WORKLOAD = ("70k-bus seeded synthetic grid (70,000 buses, 88,000 branches, 7,000 PV, 50,000 PQ loads, "
            "3,000 shunts, 12% transformers), reduced polar formulation, FP64, {} perturbed states")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--e2e-steps", type=int, default=20)
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--profile", action="store_true",
                   help="only run warmup + steps evaluations of the workload (for ncu), no timing")
    p.add_argument("--tile", type=int, default=0, help="profile mode: tile_inc (0: autotune)")
    p.add_argument("--ctas", type=int, default=0, help="profile mode: CTAs per SM")
    p.add_argument("--states", type=int, default=48,
                   help="70k workload: states evaluated per batched launch (48 = the headline configuration)")
    p.add_argument("--no-extra", action="store_true",
                   help="70k line only: skip the compact lines of the other workloads ('extra')")
    p.add_argument("--workload", default="70k",
                   choices=["70k", "contingency", "adjoint", "mixed", "extended", "newton"],
                   help="70k: the headline line (default); the others measure the batched-contingency, "
                        "adjoint and mixed-scenario workloads on one GPU and print their own line")
    return p.parse_args()


def run_profile(args):
    """A few plain evaluations of the bench workload (the batched 48-state
    launch), for an ncu capture."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_11880_gb300 import Context
    sys_ = gridgen.grid_70k()
    ctx = Context([sys_], "reduced", instances=[(0, -1)] * N_STATES)
    X = torch.from_numpy(np.concatenate([gridgen.perturbed_state(sys_, k)
                                         for k in range(1, N_STATES + 1)])).cuda()
    F, V = ctx.empty_f(), ctx.empty_vals()
    if args.tile:
        ctx.set_tuning(args.tile, args.ctas)
    else:
        ctx.autotune(X, F, V)
    print("tuning", ctx.tuning())
    for k in range(args.warmup + args.steps):
        ctx.residual_jacobian(X, F, V)
    torch.cuda.synchronize()
    ctx.check_device()
    print(f"profile run: {args.warmup + args.steps} batched evaluations of {N_STATES} states")
    return 0


def max_over_ranks(seconds, distributed, device):
    """The slowest rank's time (the timing every rank reports is its own
    CUDA-event time; the whole job's time is the maximum)."""
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    if distributed:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, units_per_rank, t_max):
    """Whole-job throughput of `world` replicas that each processed
    `units_per_rank` units, the slowest in t_max seconds."""
    return world * units_per_rank / t_max


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# algorithmic work per launch / evaluation
# --------------------------------------------------------------------------

def algorithmic_bytes(d, n_pv, n_load, n_shunt):
    """Bytes the evaluation must move at least: read the state (theta, V),
    the branch parameters (from, to: int32; r, x, b, tap, shift: FP64), the
    PQ / PV / shunt models (bus int32 + 2 or 1 FP64 each), write F and J."""
    n, m = d.n_bus, d.n_branch
    read = 16 * n + m * (8 + 5 * 8) + n_load * 20 + n_pv * 12 + n_shunt * 20
    write = 8 * (d.n_f + d.nnz)
    return read + write


def l2_note(step_bytes):
    """How the timed region relates to the 129 MB L2 (the timing rule: inputs
    larger than L2, or a flush between steps)."""
    if step_bytes > 129e6:
        return f"inputs larger than L2: every state's own x, F and J ({step_bytes / 1e6:.0f} MB) per step, no flush"
    return (f"x, F and J of the step ({step_bytes / 1e6:.0f} MB) fit in L2, so steps after the first may hit it: "
            "a batch-size sweep point, not the headline configuration")


def hbm_roofline(bytes_alg, kernel_ms, step_s, peaks, peak_kind, traffic):
    """The roofline of the dominant kernel against the measured HBM copy rate:
    achieved = the step's algorithmic bytes (read the state, the branch and
    model parameters, write F and J) over k_tile's own CUDA-event time, and
    the same bytes over the whole step (k_phasor_fx + k_tile) beside it."""
    ach = bytes_alg / (kernel_ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": "k_tile", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": ach / peaks["hbm_gbs"], "peak_kind": f"{peak_kind} copy peak (MEASURED_PEAKS.json hbm_gbs)",
            "traffic": traffic.get("dram_bytes_per_launch") if traffic else None,
            "algorithmic_bytes": bytes_alg, "kernel_ms": kernel_ms,
            "step_achieved_gbs": bytes_alg / step_s / 1e9, "step_frac": bytes_alg / step_s / 1e9 / peaks["hbm_gbs"]}


def compact_line(r):
    """The fields of a workload's line kept in the headline line's 'extra'."""
    roof = r["roofline"]
    out = {"metric": r["metric"], "value": r["value"], "unit": r["unit"], "ms_per_step": r["ms_per_step"],
           "roofline": {k: roof[k] for k in ("bound", "kernel", "frac", "step_frac", "achieved", "unit",
                                             "kernel_ms")},
           "clocks": r["clocks"], "tuning": r.get("config", {}).get("tuning")}
    if "fp64" in roof:
        out["roofline"]["fp64_k_tile_frac"] = roof["fp64"]["k_tile_frac"]
    if "breakdown" in r:
        out["breakdown"] = r["breakdown"]
    return out


def fp64_view(ops_tile, ops_phasor, kernel_ms, step_s, dev):
    """FP64-pipe operations of a launch against the FP64 FMA rate measured in
    this run by the library's pf_fp64_peak (the pair terms run on the integer
    pipe, so this is a secondary view)."""
    from paper_2011_11880_gb300 import fp64_peak
    peak, _ = fp64_peak(dev.index if dev.index is not None else 0)
    return {"executed_ops_k_tile": ops_tile, "executed_ops_step": ops_tile + ops_phasor,
            "peak_gops": peak, "peak_kind": "measured in this run by pf_fp64_peak (FP64 FMA chains)",
            "k_tile_frac": ops_tile / (kernel_ms * 1e-3) / 1e9 / peak,
            "step_frac": (ops_tile + ops_phasor) / step_s / 1e9 / peak}


def fp64_ops(d, pattern):
    """FP64-pipe operations of one instance's F and J evaluation (an FMA, a
    multiply, an add or a conversion each count one).  k_tile forms the pair
    terms in fixed point on the integer pipe; the FP64 pipe converts each
    off-diagonal value of a pair to double (one conversion), and each bus takes
    the two exact bus sums to double (2; V_o is converted exactly on the integer
    pipe), V_o^2, V_o^2 A^ - S_X, V_o^2 C^ + S_Y and the two F rows (5), plus two
    FMAs and two multiplies for the diagonal V values where the bus has a V
    column (4).  k_phasor_fx forms 1/V_o (3 FMAs after the hardware's
    reciprocal estimate) for every bus.  Returns (k_tile, k_phasor_fx)."""
    n = d.n_bus
    nnz = int(pattern[0][-1])
    if d.formulation == 0:                   # reduced: P rows of the n - 1 non-slack buses, Q rows of the PQ buses
        n_pq = d.n_f - (n - 1)
        n_diag = (n - 1) + 3 * n_pq          # (P, theta_o) of each; (P, V_o), (Q, theta_o), (Q, V_o) of a PQ bus
        n_vbus = n_pq
    else:                                    # extended: four diagonal entries per bus, and the generator rows
        n_gen = d.n_x - 2 * n - 1
        n_diag = 4 * n + 1 + n_gen + 2 * n_gen + 1   # P_s, Q_g columns, g_V rows, g_theta
        n_vbus = n
    return (nnz - n_diag) + 7 * n + 4 * n_vbus, 3 * n


def _oracle_share(kind, idx, seconds, barrier, queue):
    """One host process of the batched CPU baseline: generates its share of the
    instances (idx), meets the other processes at the barrier, then runs the
    oracle over its share cyclically for `seconds` (contingency: F + J of the
    instance with its outage; mixed: F + J + the VJP with v = F)."""
    try:
        import oracle
        if kind == "contingency":
            grids, insts = gridgen.contingency_batch(only=idx)

            def one(ins):
                sk = grids[ins.grid].copy()
                sk.br_status = sk.br_status.copy()
                sk.br_status[ins.outage] = 0
                oracle.residual(sk, ins.x)
                oracle.jacobian(sk, ins.x)
        else:
            grids, insts = gridgen.mixed_batch(only=idx)

            def one(ins):
                sk = grids[ins.grid]
                f = oracle.residual(sk, ins.x, p_inj=ins.p_inj, q_inj=ins.q_inj)
                oracle.jacobian(sk, ins.x)
                oracle.vjp(sk, ins.x, f)
        barrier.wait(timeout=600)
        t0, m = time.perf_counter(), 0
        while time.perf_counter() - t0 < seconds:
            one(insts[m % len(insts)])
            m += 1
        queue.put((m, time.perf_counter() - t0, ""))
    except Exception as e:  # reported by the parent
        queue.put((0, 0.0, f"{type(e).__name__}: {e}"))


def oracle_pool(kind, n_inst, seconds):
    """The oracle on every host core at once, one process per core, each on its
    own share of the instances (the one-instance-per-core deployment the paper
    recommends for many independent cases).  Processes are spawned, not forked
    (the parent holds a CUDA context).  Returns (instances/s, instances,
    seconds, processes)."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    threads = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {var: os.environ.get(var) for var in threads}
    ctx = mp.get_context("spawn")
    barrier, queue = ctx.Barrier(cores), ctx.Queue()
    procs = [ctx.Process(target=_oracle_share, args=(kind, list(range(w, n_inst, cores)), seconds, barrier, queue))
             for w in range(cores)]
    try:
        for var in threads:
            os.environ[var] = "1"                   # one thread per process (read by the children)
        for pr in procs:
            pr.start()
    finally:
        for var, val in saved.items():
            if val is None:
                os.environ.pop(var, None)
            else:
                os.environ[var] = val
    import queue as queue_mod
    res, deadline = [], time.time() + seconds + 900
    try:
        while len(res) < len(procs):
            try:
                res.append(queue.get(timeout=1.0))
            except queue_mod.Empty:
                if any(pr.exitcode not in (None, 0) for pr in procs) or \
                        all(pr.exitcode is not None for pr in procs):
                    raise RuntimeError("an oracle process exited without a result")
                if time.time() > deadline:
                    raise RuntimeError("the oracle processes did not finish")
    finally:
        for pr in procs:                            # our own children, by handle
            if pr.is_alive() and len(res) < len(procs):
                pr.terminate()
            pr.join(timeout=60)
    errors = [r[2] for r in res if r[2]]
    if errors:
        raise RuntimeError("oracle process failed: " + errors[0])
    m = sum(r[0] for r in res)
    el = max(r[1] for r in res)
    return m / el, m, el, cores


def host_cpu():
    """The host the oracle ran on: architecture, model name where the OS gives one, logical CPUs."""
    import platform
    model = ""
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.lower().startswith(("model name", "cpu model")):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    cpus = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return f"{platform.machine()}{', ' + model if model else ''}, {cpus} logical CPUs"


def launches_per_eval(ctx):
    """Kernels one evaluation of the context launches: k_phasor_fx and k_tile,
    and k_fused_large where a bus has more than 32 neighbours."""
    return 2 + (1 if ctx.dims.max_degree > 32 else 0)


def source_hash():
    """Hash of the code (comments and blank space removed) of the sources that
    decide k_tile's memory traffic: the kernel and the data layout."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in ("pf_eval.cu", "pf_build.cu", "pf_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2011_11880_gb300", "csrc", f)) as fh:
            code = fh.read()
        code = re.sub(r"/\*.*?\*/", " ", code, flags=re.S)
        code = re.sub(r"//[^\n]*", " ", code)
        h.update(" ".join(code.split()).encode())
    return h.hexdigest()[:16]


# --------------------------------------------------------------------------
# reference arm: the CPU oracle on the host cores
# --------------------------------------------------------------------------

def time_oracle(sys_, states, seconds, reduced=True):
    import oracle
    t0 = time.perf_counter()
    n = 0
    while True:
        x = states[n % len(states)]
        oracle.residual(sys_, x)
        oracle.jacobian(sys_, x)
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds or n >= 1000:
            return n / el, n, el


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    sys_ = gridgen.grid_70k()
    states = [gridgen.perturbed_state(sys_, k) for k in range(1, N_STATES + 1)]
    total_steps = args.warmup + args.steps
    budget = min(max(args.cpu_seconds, 5.0), 120.0)
    rate, n, el = time_oracle(sys_, states, budget)
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": "evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / rate,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD.format(N_STATES), "sample": f"{n} oracle F+J evaluations"},
        "e2e": {"value": rate, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "cpu_baseline": {"value": rate, "unit": "evals/s", "cores": 1, "kind": "oracle", "host": host_cpu(),
                         "sample": f"{n} F+J evaluations of the 70k grid ({el:.1f} s, numpy FP64, "
                                   f"one thread; requested {total_steps} steps bounded to {budget:.0f} s)"},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------

def main():
    global N_STATES
    args = parse()
    if args.states < 1:
        raise SystemExit("--states must be positive")
    N_STATES = args.states
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.profile:
        return run_profile(args)
    if args.workload != "70k":
        return run_workload(args)
    if args.impl == "reference":
        if world > 1 and "RANK" in os.environ:
            world = int(os.environ["WORLD_SIZE"])
        return run_reference(args, rank, max(world, 1))

    import torch
    import torch.distributed as dist

    distributed = "RANK" in os.environ and int(os.environ.get("WORLD_SIZE", "1")) > 1
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if distributed:
        dist.init_process_group("nccl", device_id=dev)
    world = dist.get_world_size() if distributed else 1

    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_11880_gb300 import Context

    sys_ = gridgen.grid_70k()
    states_np = [gridgen.perturbed_state(sys_, k) for k in range(1, N_STATES + 1)]

    def capture(fn):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            fn()
        return g

    stream = torch.cuda.Stream(device=dev)
    lead = torch.empty(LEAD_BYTES // 4, dtype=torch.float32, device=dev)

    # ---- batched: the states as instances of the grid, one launch per step ----
    ctx = Context([sys_], "reduced", instances=[(0, -1)] * N_STATES)
    d = ctx.dims
    one = Context(sys_, "reduced")            # single-instance context for the comparison
    d1 = one.dims
    X = torch.from_numpy(np.concatenate(states_np)).to(dev)
    F = torch.empty(d.n_f, dtype=torch.float64, device=dev)
    V = torch.empty(d.nnz, dtype=torch.float64, device=dev)
    with torch.cuda.stream(stream):
        tuning = ctx.autotune(X, F, V)
        ctx.residual_jacobian(X, F, V)
        torch.cuda.synchronize()
        g_eval = capture(lambda: ctx.residual_jacobian(X, F, V))
        # (with fuse_phasor the fused stage forms its records: no phasor stage to replay)
        g_ph = None if tuning.get("fuse_phasor") else capture(lambda: ctx.eval_stage(1, X, F, V))
        g_fu = capture(lambda: ctx.eval_stage(2, X, F, V))
    torch.cuda.synchronize()

    K, W = args.steps, max(args.warmup, 3)
    with torch.cuda.stream(stream):
        for k in range(W):
            g_eval.replay()
    torch.cuda.synchronize()
    if distributed:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    sampler.start()
    time.sleep(0.3)
    ev_a, ev_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    wall0 = time.perf_counter()
    torch.cuda.nvtx.range_push("bench_timed")
    with torch.cuda.stream(stream):
        ev_a.record(stream)
        for k in range(K):
            g_eval.replay()
        ev_b.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    wall = time.perf_counter() - wall0
    if distributed:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    t_sum = ev_a.elapsed_time(ev_b) / 1000.0
    t_max = max_over_ranks(t_sum, distributed, dev)
    value = job_throughput(world, K * N_STATES, t_max)
    ms_per_step = 1000.0 * t_max / K

    # ---- the dominant kernel alone: the batched k_tile launch between events ----
    KF = min(K, 200)
    with torch.cuda.stream(stream):
        if g_ph is not None:
            g_ph.replay()
        ev_a.record(stream)
        for k in range(KF):
            g_fu.replay()
        ev_b.record(stream)
    torch.cuda.synchronize()
    kf_ms = ev_a.elapsed_time(ev_b) / KF

    # ---- single instance, one evaluation at a time (each state its own x, F, J) ----
    Xs = X.view(N_STATES, d1.n_x)
    Fs = torch.empty(N_STATES, d1.n_f, dtype=torch.float64, device=dev)
    Vs = torch.empty(N_STATES, d1.nnz, dtype=torch.float64, device=dev)
    with torch.cuda.stream(stream):
        one_tuning = one.autotune(Xs[0], Fs[0], Vs[0])
        for k in range(N_STATES):
            one.residual_jacobian(Xs[k], Fs[k], Vs[k])
        torch.cuda.synchronize()
        # one graph holding the 48 evaluations one after the other (each its own launches),
        # so the host's graph-launch rate does not bound the GPU's one-at-a-time rate
        g_one = capture(lambda: [one.residual_jacobian(Xs[k], Fs[k], Vs[k]) for k in range(N_STATES)])
    torch.cuda.synchronize()
    KS = max(1, min(K, 20000 // N_STATES))
    with torch.cuda.stream(stream):
        lead.fill_(1.0)
        ev_a.record(stream)
        for k in range(KS):
            g_one.replay()
        ev_b.record(stream)
    torch.cuda.synchronize()
    single_rate = KS * N_STATES / (ev_a.elapsed_time(ev_b) / 1000.0)

    # ---- end to end through the host-buffer entry point (one batched step) ----
    E = min(args.e2e_steps, K)
    xh = torch.from_numpy(np.concatenate(states_np)).pin_memory().numpy()
    Fh = torch.empty(d.n_f, dtype=torch.float64).pin_memory().numpy()
    Vh = torch.empty(d.nnz, dtype=torch.float64).pin_memory().numpy()
    with torch.cuda.stream(stream):
        for k in range(2):
            ctx.residual_jacobian_host(xh, Fh, Vh, stream=stream)
        stream.synchronize()
        t0 = time.perf_counter()
        for k in range(E):
            ctx.residual_jacobian_host(xh, Fh, Vh, stream=stream)
        e2e_t = time.perf_counter() - t0
    e2e_value = job_throughput(world, E * N_STATES, max_over_ranks(e2e_t, distributed, dev))

    # ---- the timed outputs equal single-instance evaluations ----
    for k in (0, N_STATES - 1):
        assert torch.equal(F[ctx.f_off[k]:ctx.f_off[k + 1]], Fs[k]), "batched F differs from single instance"
        assert torch.equal(V[ctx.nnz_off[k]:ctx.nnz_off[k + 1]], Vs[k]), "batched J differs from single instance"
    ctx.check_device()
    one.check_device()

    peaks, peak_kind = load_peaks()
    n_pv, n_load, n_shunt = sys_.n_pv, sys_.load_bus.shape[0], sys_.sh_bus.shape[0]
    pattern = one.pattern()
    fp_kf, fp_ph = fp64_ops(d1, pattern)
    bytes_alg = N_STATES * algorithmic_bytes(d1, n_pv, n_load, n_shunt)   # one batched step
    eval_s = t_max / K                                                       # one batched step
    roofline = hbm_roofline(bytes_alg, kf_ms, eval_s, peaks, peak_kind, load_traffic())
    roofline["fp64"] = fp64_view(N_STATES * fp_kf, N_STATES * fp_ph, kf_ms, eval_s, dev)

    cpu = None
    if rank == 0:
        rate, n, el = time_oracle(sys_, states_np, args.cpu_seconds)
        cpu = {"value": rate, "unit": "evals/s", "cores": 1, "kind": "oracle", "host": host_cpu(),
               "sample": f"{n} F+J evaluations of the 70k grid in {el:.1f} s (numpy FP64, one thread)"}

    line = {
        "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD.format(N_STATES), "n_f_per_state": d1.n_f, "nnz_per_state": d1.nnz,
                   "step": f"one batched launch over {N_STATES} states (instances of the grid)",
                   "l2": l2_note(N_STATES * 8 * (d1.n_x + d1.n_f + d1.nnz)),
                   "tuning": tuning, "timed_region_wall_s": wall, "parallelism": f"replicas x{world}"},
        "single_instance": {"value": single_rate, "unit": "evals/s", "tuning": one_tuning,
                            "how": ("one launch per evaluation (k_tile forming its voltage records)"
                                    if one_tuning.get("fuse_phasor") else
                                    "one launch pair per evaluation (k_phasor_fx, k_tile)")
                                   + f", {N_STATES} states with their own buffers evaluated one after the other "
                                     "from one CUDA graph"},
        "batched_over_single": value / world / single_rate,
        "e2e": {"value": e2e_value, "unit": "evals/s", "h2d_bytes_per_step": 8 * d.n_x,
                "d2h_bytes_per_step": 8 * (d.n_f + d.nnz), "steps": E},
        "gpu_launches": launches_per_eval(ctx) * K,
        "roofline": roofline,
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    ctx.close()
    one.close()
    if not distributed and not args.no_extra:
        # the other workloads on the same GPU, compact: value, time, roofline fractions, clocks
        KX = max(1, min(K, 20))
        line["extra"] = {}
        # (a failing extra workload is reported in its key; the headline line is printed regardless)
        for name, fn in (("extended_70k", measure_extended), ("contingency", measure_contingency),
                         ("adjoint_70k_64cot", measure_adjoint), ("mixed", measure_mixed)):
            try:
                line["extra"][name] = compact_line(fn(torch, stream, KX, 3))
            except Exception as exc:                  # noqa: BLE001
                line["extra"][name] = {"error": f"{type(exc).__name__}: {exc}"}
        # Newton power flow at the paper's four grid sizes (outside the hot path; host-timed)
        try:
            nt = measure_newton(argparse.Namespace(steps=1, cpu_seconds=0.0))
            line["extra"]["newton"] = {"metric": nt["metric"], "value": nt["value"], "unit": nt["unit"],
                                       "runs": [{k: r[k] for k in ("n_bus", "case", "method", "solver", "seconds",
                                                                   "iterations", "converged", "max_mismatch")}
                                                for r in nt["runs"]]}
        except Exception as exc:                      # noqa: BLE001
            line["extra"]["newton"] = {"error": f"{type(exc).__name__}: {exc}"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if distributed:
        dist.destroy_process_group()
    return 0


# --------------------------------------------------------------------------
# the other workloads (one GPU each; not the headline line)
# --------------------------------------------------------------------------

def _graph(torch, stream, fn):
    with torch.cuda.stream(stream):
        fn()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            fn()
    torch.cuda.synchronize()
    return g


def _time_graph(torch, stream, g, reps):
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        g.replay()
        a.record(stream)
        for _ in range(reps):
            g.replay()
        b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1000.0 / reps


def run_workload(args):
    """One of the other workloads on one GPU, printed as its own line with the
    oracle's CPU baseline beside it (see the measure_* functions)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    stream = torch.cuda.Stream()
    K, W = min(max(args.steps, 1), 200), max(args.warmup, 3)
    out = {"n_gpus": 1, "steps": K, "warmup": W, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "ours"}
    if args.workload == "newton":
        out.update(measure_newton(args))
        print(json.dumps(out), flush=True)
        return 0
    fn = {"contingency": measure_contingency, "adjoint": measure_adjoint, "mixed": measure_mixed,
          "extended": measure_extended}[args.workload]
    res = fn(torch, stream, K, W, cpu_seconds=args.cpu_seconds)
    out.update(res)
    print(json.dumps(out), flush=True)
    return 0


def _clocked(torch, stream, g, K):
    """Times K replays of graph g with CUDA events while nvidia-smi samples the
    clocks; returns (seconds per replay, clock record)."""
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    torch.cuda.nvtx.range_push("bench_timed")
    t = _time_graph(torch, stream, g, K)
    torch.cuda.nvtx.range_pop()
    return t, sampler.stop()


def measure_contingency(torch, stream, K, W, cpu_seconds=0.0):
    """2,048 x 2,000-bus + 256 x 10,000-bus instances, one seeded branch outage
    each (reduced formulation, one masked launch pair per step)."""
    from paper_2011_11880_gb300 import Context
    peaks, peak_kind = load_peaks()
    grids, insts = gridgen.contingency_batch()
    ctx = Context(grids, instances=[(i.grid, i.outage) for i in insts])
    X = torch.from_numpy(np.concatenate([i.x for i in insts])).cuda()
    F, V = ctx.empty_f(), ctx.empty_vals()
    with torch.cuda.stream(stream):
        tuning = ctx.autotune(X, F, V, stream=stream)
    g = _graph(torch, stream, lambda: ctx.residual_jacobian(X, F, V, stream=stream))
    gp = None if tuning.get("fuse_phasor") else _graph(torch, stream, lambda: ctx.eval_stage(1, X, F, V, stream=stream))
    gf = _graph(torch, stream, lambda: ctx.eval_stage(2, X, F, V, stream=stream))
    for _ in range(W):
        g.replay()
    t, clocks = _clocked(torch, stream, g, K)
    if gp is not None:
        gp.replay()
    kf = _time_graph(torch, stream, gf, K)
    n = len(insts)
    bytes_alg = 0
    for gi, gsys in enumerate(grids):
        cnt = sum(1 for i in insts if i.grid == gi)
        one = Context(gsys)
        bytes_alg += cnt * algorithmic_bytes(one.dims, gsys.n_pv, gsys.load_bus.shape[0], gsys.sh_bus.shape[0])
        one.close()
    ctx.check_device()
    res = {"metric": "instance F+J evals/s, batched contingencies", "value": n / t, "unit": "evals/s",
           "ms_per_step": 1e3 * t,
           "config": {"workload": "2,048 x 2,000-bus + 256 x 10,000-bus seeded synthetic grids, one seeded branch "
                                  "outage per instance, reduced formulation, one launch pair",
                      "n_f": ctx.dims.n_f, "nnz": ctx.dims.nnz, "tuning": tuning,
                      "l2": "inputs larger than L2 (x, F, J of 2,304 instances: 1 GB)"},
           "roofline": hbm_roofline(bytes_alg, 1e3 * kf, t, peaks, peak_kind, None),
           "breakdown": {"k_tile_ms": 1e3 * kf}, "clocks": clocks,
           "gpu_launches": launches_per_eval(ctx) * K}
    ctx.close()
    if cpu_seconds > 0:
        cpu_rate, m, el, cores = oracle_pool("contingency", n, cpu_seconds)
        res["cpu_baseline"] = {"value": cpu_rate, "unit": "evals/s", "cores": cores, "kind": "oracle",
                               "host": host_cpu(),
                               "sample": f"{m} instance F+J evaluations in {el:.1f} s, one process per host core "
                                         f"({cores}), each cycling over its 1/{cores} of the 2,304 instances"}
    return res



def measure_adjoint(torch, stream, K, W, cpu_seconds=0.0):
    """The 70k grid with 64 seeded Gaussian cotangents, every gradient
    (theta, V, P_inj, Q_inj, r, x, b_c, tau), one pf_vjp call per step."""
    import oracle
    from paper_2011_11880_gb300 import Context
    peaks, peak_kind = load_peaks()
    sys_ = gridgen.grid_70k()
    ctx = Context(sys_)
    B = 64
    x = torch.from_numpy(gridgen.perturbed_state(sys_, 1)).cuda()
    Vn = gridgen.gaussian_cotangents(ctx.dims.n_f, B)
    V = torch.from_numpy(Vn).cuda().reshape(-1)
    g = _graph(torch, stream, lambda: ctx.vjp(x, V, B, stream=stream))
    for _ in range(W):
        g.replay()
    t, clocks = _clocked(torch, stream, g, K)
    breakdown = {}
    for name, want in (("state", ("x",)), ("branch_params", ("br_r", "br_x", "br_b", "br_tap")),
                       ("injections", ("p_inj", "q_inj"))):
        gw = _graph(torch, stream, lambda want=want: ctx.vjp(x, V, B, want=want, stream=stream))
        breakdown[name + "_ms"] = 1e3 * _time_graph(torch, stream, gw, K)
    d = ctx.dims
    # per cotangent: read v, write the gradients; x and the parameters once
    bytes_alg = B * 8 * (d.n_f + d.n_x + 2 * d.n_bus_inst + 4 * d.n_branch_inst) + \
        algorithmic_bytes(d, sys_.n_pv, sys_.load_bus.shape[0], sys_.sh_bus.shape[0]) - 8 * (d.n_f + d.nnz)
    ctx.check_device()
    roof = hbm_roofline(bytes_alg, 1e3 * t, t, peaks, peak_kind, None)
    roof["kernel"] = "pf_vjp (one call: transpose, state, parameter and injection kernels)"
    res = {"metric": "VJPs/s (cotangents/s), 70k grid, every gradient", "value": B / t, "unit": "cotangents/s",
           "ms_per_step": 1e3 * t,
           "config": {"workload": "70k-bus seeded synthetic grid, 64 Gaussian cotangents (seeds 4000+k), "
                                  "v^T dF/d(theta, V, P_inj, Q_inj, r, x, b_c, tau), one call"},
           "roofline": roof, "breakdown": breakdown, "clocks": clocks, "gpu_launches": 5 * K}
    ctx.close()
    if cpu_seconds > 0:
        xn = gridgen.perturbed_state(sys_, 1)
        t0, m = time.perf_counter(), 0
        while time.perf_counter() - t0 < cpu_seconds and m < B:
            oracle.vjp(sys_, xn, Vn[m])
            m += 1
        el = time.perf_counter() - t0
        res["cpu_baseline"] = {"value": m / el, "unit": "cotangents/s", "cores": 1, "kind": "oracle",
                               "host": host_cpu(), "sample": f"{m} oracle VJPs in {el:.1f} s"}
    return res


def measure_mixed(torch, stream, K, W, cpu_seconds=0.0):
    """4,096 grids of 500-20,000 buses (log-uniform), PV output and load scaled
    per instance (injection overrides): F + J, then v^T dF/d(x, P_inj, Q_inj)
    with v = F, in one captured iteration."""
    from paper_2011_11880_gb300 import Context
    peaks, peak_kind = load_peaks()
    grids, insts = gridgen.mixed_batch()
    ctx = Context(grids, instances=[(k, -1) for k in range(len(grids))])
    X = torch.from_numpy(np.concatenate([i.x for i in insts])).cuda()
    Pi = torch.from_numpy(np.concatenate([i.p_inj for i in insts])).cuda()
    Qi = torch.from_numpy(np.concatenate([i.q_inj for i in insts])).cuda()
    F, V = ctx.empty_f(), ctx.empty_vals()
    with torch.cuda.stream(stream):
        tuning = ctx.autotune(X, F, V, stream=stream)
    keep = {}

    def iteration():
        ctx.eval(X, F, V, stream=stream, p_inj=Pi, q_inj=Qi)
        keep["g"] = ctx.vjp(X, F, 1, want=("x", "p_inj", "q_inj"), stream=stream, p_inj=Pi, q_inj=Qi)

    g = _graph(torch, stream, iteration)
    for _ in range(W):
        g.replay()
    t, clocks = _clocked(torch, stream, g, K)
    gfj = _graph(torch, stream, lambda: ctx.eval(X, F, V, stream=stream, p_inj=Pi, q_inj=Qi))
    fj = _time_graph(torch, stream, gfj, K)
    d = ctx.dims
    n = len(insts)
    # F + J: the state, parameters and injection overrides read, F and J written;
    # VJP: v = F read, the x, P_inj and Q_inj gradients written
    n_branch = sum(int(gg.br_from.shape[0]) for gg in grids)
    n_load = sum(int(gg.load_bus.shape[0]) for gg in grids)
    n_pv = sum(int(gg.n_pv) for gg in grids)
    n_sh = sum(int(gg.sh_bus.shape[0]) for gg in grids)
    nb = d.n_bus_inst
    fj_bytes = 16 * nb + 48 * n_branch + 20 * n_load + 12 * n_pv + 20 * n_sh + 16 * nb + 8 * (d.n_f + d.nnz)
    vjp_bytes = 8 * d.n_f + 8 * (d.n_x + 2 * nb)
    ctx.check_device()
    roof = hbm_roofline(fj_bytes + vjp_bytes, 1e3 * t, t, peaks, peak_kind, None)
    roof["kernel"] = "the whole iteration (F + J, then the VJP)"
    res = {"metric": "instance iterations/s (F+J, then J^T F), mixed scenarios", "value": n / t,
           "unit": "iterations/s", "ms_per_step": 1e3 * t,
           "config": {"workload": "4,096 seeded synthetic grids of 500-20,000 buses (log-uniform), "
                                  "PV output x U[0.5,1.5], load x U[0.8,1.2] as injection overrides, "
                                  "F + J then v^T dF/d(x, P_inj, Q_inj) with v = F, one captured graph",
                      "buses": int(nb), "tuning": tuning},
           "roofline": roof, "breakdown": {"fj_ms": 1e3 * fj, "vjp_ms": 1e3 * (t - fj)}, "clocks": clocks,
           "gpu_launches": (launches_per_eval(ctx) + 5) * K}
    ctx.close()
    if cpu_seconds > 0:
        cpu_rate, m, el, cores = oracle_pool("mixed", n, cpu_seconds)
        res["cpu_baseline"] = {"value": cpu_rate, "unit": "iterations/s", "cores": cores, "kind": "oracle",
                               "host": host_cpu(),
                               "sample": f"{m} instance iterations in {el:.1f} s, one process per host core "
                                         f"({cores}), each cycling over its 1/{cores} of the 4,096 instances"}
    return res



def measure_extended(torch, stream, K, W, cpu_seconds=0.0):
    """The 70k grid in the paper's extended formulation (Sec. II-A, Eqs. 1-3:
    rows g_p, g_q of every bus, g_V of every generator, g_theta; columns theta,
    V, Q_g, P_s), 48 states per launch, as the headline's batched step."""
    from paper_2011_11880_gb300 import Context
    peaks, peak_kind = load_peaks()
    sys_ = gridgen.grid_70k()
    S = 48
    one = Context(sys_, "extended")
    d1 = one.dims
    xs = [gridgen.perturbed_state(sys_, k, extended=True) for k in range(1, S + 1)]
    ctx = Context([sys_], "extended", instances=[(0, -1)] * S)
    X = torch.from_numpy(np.concatenate(xs)).cuda()
    F, V = ctx.empty_f(), ctx.empty_vals()
    with torch.cuda.stream(stream):
        tuning = ctx.autotune(X, F, V, stream=stream)
    g = _graph(torch, stream, lambda: ctx.residual_jacobian(X, F, V, stream=stream))
    gp = None if tuning.get("fuse_phasor") else _graph(torch, stream, lambda: ctx.eval_stage(1, X, F, V, stream=stream))
    gf = _graph(torch, stream, lambda: ctx.eval_stage(2, X, F, V, stream=stream))
    for _ in range(W):
        g.replay()
    t, clocks = _clocked(torch, stream, g, K)
    if gp is not None:
        gp.replay()
    kf = _time_graph(torch, stream, gf, K)
    bytes_alg = S * (algorithmic_bytes(d1, sys_.n_pv, sys_.load_bus.shape[0], sys_.sh_bus.shape[0])
                     + 8 * (d1.n_x - 2 * d1.n_bus))          # the Q_g and P_s entries of x
    fp_kf, fp_ph = fp64_ops(d1, one.pattern())
    roof = hbm_roofline(bytes_alg, 1e3 * kf, t, peaks, peak_kind, None)
    roof["fp64"] = fp64_view(S * fp_kf, S * fp_ph, 1e3 * kf, t, X.device)
    ctx.check_device()
    res = {"metric": "F+J evals/s on 70k-bus grid, extended formulation (batched)", "value": S / t,
           "unit": "evals/s", "ms_per_step": 1e3 * t,
           "config": {"workload": "70k-bus seeded synthetic grid, extended formulation (Eqs. 1-3), 48 perturbed "
                                  "states per launch", "n_f_per_state": d1.n_f, "nnz_per_state": d1.nnz,
                      "tuning": tuning},
           "roofline": roof, "clocks": clocks, "gpu_launches": launches_per_eval(ctx) * K}
    ctx.close()
    one.close()
    return res



def _finite(info):
    """A solver's info with non-finite numbers (a diverged run's mismatch) as null."""
    return {k: (None if isinstance(v, float) and not math.isfinite(v) else v) for k, v in info.items()}


def constructed_case(n_bus, seed):
    """A synthetic grid with a known power-flow solution: the point drawn by
    gridgen.target_state, and per-bus injections equal to the network's own
    flows there, evaluated by this library (the extended formulation's g_p,
    g_q rows at zero injections, Q_g = P_s = 0)."""
    import torch
    from paper_2011_11880_gb300 import Context
    g = gridgen.grid_70k() if n_bus == 70000 else gridgen.synthetic_grid(n_bus, seed)
    th, V = gridgen.target_state(g, seed + 1)
    n = g.n_bus
    z = np.zeros(n)
    g0 = gridgen.with_injections(g, z, z, V)
    ctx = Context(g0, "extended")
    x = np.zeros(gridgen.state_size(g0, True))
    x[:n], x[n:2 * n] = th, V
    F = ctx.residual(torch.from_numpy(x).cuda()).cpu().numpy()
    ctx.close()
    return gridgen.with_injections(g, F[:n], F[n:2 * n], V)


def measure_newton(args):
    """Flat-start Newton power flow and fast decoupled iterations (F, J, the
    convergence test and the update in this library's kernels; the sparse
    solve in cuSOLVER), timed on the host around each solve, on grids of the
    four sizes of the paper's Newton comparison (2,000 to 70,000 buses)."""
    import torch
    import oracle
    from paper_2011_11880_gb300 import Context
    # The ring-of-meshes grids have a flat-start Newton solution from their drawn loads only at
    # light load (2,000 buses x 0.2, 10,000 x 0.1; a CPU sparse Newton agrees), and none at
    # 25,000 or 70,000 buses: the losses the single slack must cover travel the whole ring.
    # Those two sizes use a constructed case (constructed_case) whose solution is known.
    cases = [(2000, "drawn loads x 0.2", lambda: gridgen.synthetic_grid(2000, 3000, load_scale=0.2), ("lu", "qr")),
             (10000, "drawn loads x 0.1", lambda: gridgen.synthetic_grid(10000, 3001, load_scale=0.1), ("lu", "qr")),
             (25000, "constructed", lambda: constructed_case(25000, 2500), ("lu",)),
             (70000, "constructed", lambda: constructed_case(70000, 2500), ("lu",))]
    runs = []
    for n_bus, kind, make, solvers in cases:
        sk = make()
        for solver in solvers:
            ctx = Context(sk)
            ctx.set_newton_solver(solver)
            x0 = torch.from_numpy(gridgen.flat_state(sk)).cuda()
            x = x0.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            first = ctx.newton(x, tol=1e-8, max_iter=15)          # includes the first (host) LU
            t_first = time.perf_counter() - t0
            ts = []
            for _ in range(max(1, min(args.steps, 3))):
                x.copy_(x0)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                info = ctx.newton(x, tol=1e-8, max_iter=15)
                ts.append(time.perf_counter() - t0)
            runs.append({"n_bus": n_bus, "case": kind, "method": "newton", "solver": solver,
                         "seconds": float(np.median(ts)), "seconds_first_call": t_first, **_finite(info)})
            ctx.check_device()
            ctx.close()
        # fast decoupled iterations (B', B'' factored once, on the first call)
        ctx = Context(sk)
        x0 = torch.from_numpy(gridgen.flat_state(sk)).cuda()
        x = x0.clone()
        ctx.fdlf(x, tol=1e-8, max_iter=100)
        ts = []
        for _ in range(max(1, min(args.steps, 3))):
            x.copy_(x0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = ctx.fdlf(x, tol=1e-8, max_iter=100)
            ts.append(time.perf_counter() - t0)
        runs.append({"n_bus": n_bus, "case": kind, "method": "fast decoupled", "solver": "lu",
                     "seconds": float(np.median(ts)), **_finite(info)})
        ctx.check_device()
        ctx.close()
    ctx = None
    clocks = {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["not sampled (host-synchronous loop)"],
              "samples": 0}
    t = [r for r in runs if r["n_bus"] == 70000 and r["method"] == "newton" and r["solver"] == "lu"][0]["seconds"]
    s2 = gridgen.synthetic_grid(2000, 3000, load_scale=0.2)
    t0, m = time.perf_counter(), 0
    while time.perf_counter() - t0 < args.cpu_seconds and m < 3:   # (0 s: no CPU baseline)
        oracle.newton_dense(s2, gridgen.flat_state(s2), tol=1e-8)
        m += 1
    el = time.perf_counter() - t0
    return {"metric": "flat-start Newton power flow, seconds per solve (70,000-bus grid)", "value": t,
                "unit": "s", "higher_is_better": False, "ms_per_step": 1e3 * t,
                "config": {"workload": "seeded synthetic grids, reduced formulation, flat start, max |F| <= 1e-8: "
                                       "2,000 buses (drawn loads x 0.2), 10,000 (x 0.1), and 25,000 and the "
                                       "70,000-bus grid with constructed injections (the network's flows at "
                                       "theta ~ U[-0.003, 0.003], V ~ 1 + U[-0.005, 0.005])",
                           "solver": "LU refactorization (host LU of the first J, cuSOLVER-Rf on the "
                                     "device after it; later solves reuse it) and, up to 10,000 buses, "
                                     "cuSOLVER sparse QR every iteration for comparison"},
                "runs": runs, "clocks": clocks, "gpu_launches": 0,
                "cpu_baseline": {"value": el / max(m, 1), "unit": "s", "cores": 1, "kind": "oracle", "host": host_cpu(),
                                 "sample": f"{m} dense-Newton solves of the 2,000-bus grid in {el:.1f} s "
                                           "(dense LU)"}}



def load_traffic():
    """DRAM bytes per k_tile launch from the committed ncu summary, used only
    while the kernel source is the one that was profiled and for the number of
    states it was profiled with."""
    path = os.path.join(ROOT, "profiles", "k_tile_traffic_70k.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except Exception:
        return None
    if rec.get("source_sha256_16") != source_hash() or rec.get("states") != N_STATES:
        return None
    return rec


if __name__ == "__main__":
    sys.exit(main())
