"""Python face of libpf.so: a Context owns one built pattern (one or many
grids and instances); its methods pass torch device buffers and the current
CUDA stream to the C ABI.  All arithmetic runs in the library's kernels."""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import PfDims, PfGrads, PfInstance, PfNewtonInfo, PfOverrides, PfSystem, PfTuning, check

FORMULATIONS = {"reduced": _lib.PF_REDUCED, "extended": _lib.PF_EXTENDED}


def _stream(stream=None) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t: torch.Tensor | None, dtype=torch.float64, numel: int | None = None, name: str = "tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


class _SystemArrays:
    """Keeps contiguous numpy copies alive while a PfSystem points at them."""

    def __init__(self, sys):
        def arr(name, dt):
            v = getattr(sys, name, None)
            if v is None:
                return None
            return np.ascontiguousarray(np.asarray(v, dtype=dt))

        self.a = {}
        for name in ("br_from", "br_to", "load_bus", "pv_bus", "sh_bus"):
            self.a[name] = arr(name, np.int32)
        for name in ("br_r", "br_x", "br_b", "br_tap", "br_shift", "br_g_fr", "br_g_to",
                     "load_p", "load_q", "pv_p", "pv_vset", "sh_g", "sh_b"):
            self.a[name] = arr(name, np.float64)
        self.a["br_status"] = arr("br_status", np.uint8)
        s = PfSystem()
        s.n_bus = int(sys.n_bus)
        s.n_branch = int(self.a["br_from"].shape[0])
        s.n_load = int(self.a["load_bus"].shape[0]) if self.a["load_bus"] is not None else 0
        s.n_pv = int(self.a["pv_bus"].shape[0]) if self.a["pv_bus"] is not None else 0
        s.n_shunt = int(self.a["sh_bus"].shape[0]) if self.a["sh_bus"] is not None else 0
        s.slack_bus = int(sys.slack_bus)
        s.slack_vset = float(getattr(sys, "slack_vset", 1.0))
        s.slack_theta = float(getattr(sys, "slack_theta", 0.0))
        for name, v in self.a.items():
            if v is not None and v.size > 0:
                ct = {np.int32: ctypes.c_int32, np.float64: ctypes.c_double, np.uint8: ctypes.c_uint8}[v.dtype.type]
                setattr(s, name, v.ctypes.data_as(ctypes.POINTER(ct)))
        self.struct = s


@dataclass
class Dims:
    formulation: int
    n_grids: int
    n_instances: int
    max_degree: int
    n_bus: int
    n_branch: int
    n_inc: int
    n_x: int
    n_f: int
    nnz: int
    n_bus_inst: int
    n_branch_inst: int
    n_gen_inst: int


class Context:
    """Built index maps of one or more grids.

    ``Context(system, "reduced")`` for one network; ``Context([g0, g1, ...],
    formulation, instances=[(grid, outage), ...])`` for a batch.  Systems are
    any objects with the attributes of ``pf_system`` (numpy-compatible).
    """

    def __init__(self, systems, formulation: str | int = "reduced", instances=None, stream=None):
        lib = _lib.load()
        if not isinstance(systems, (list, tuple)):
            systems = [systems]
        form = FORMULATIONS.get(formulation, formulation)
        arrays = [_SystemArrays(s) for s in systems]
        structs = (PfSystem * len(arrays))(*[a.struct for a in arrays])
        if instances is None:
            instances = [(g, -1) for g in range(len(systems))]
        inst = (PfInstance * len(instances))(*[PfInstance(int(g), int(o)) for g, o in instances])
        h = ctypes.c_void_p()
        with torch.cuda.device(torch.cuda.current_device()):
            check(lib.pf_build_batch(structs, len(arrays), inst, len(instances), int(form), _stream(stream),
                                     ctypes.byref(h)), "pf_build_batch")
        self._h = h
        self._lib = lib
        d = PfDims()
        check(lib.pf_get_dims(self._h, ctypes.byref(d)), "pf_get_dims")
        self.dims = Dims(*[getattr(d, f[0]) for f in PfDims._fields_])
        n = self.dims.n_instances + 1
        xo, fo, vo = (np.zeros(n, np.int64) for _ in range(3))
        check(lib.pf_offsets(self._h, xo.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                             fo.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                             vo.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))), "pf_offsets")
        self.x_off, self.f_off, self.nnz_off = xo, fo, vo

    # ---- lifetime ----
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.pf_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- maps ----
    def grid_sizes(self, grid: int = 0):
        nf, nnz, nx = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        check(self._lib.pf_grid_sizes(self._h, grid, ctypes.byref(nf), ctypes.byref(nnz), ctypes.byref(nx)),
              "pf_grid_sizes")
        return nf.value, nnz.value, nx.value

    def pattern(self, grid: int = 0):
        nf, nnz, _ = self.grid_sizes(grid)
        rp = np.zeros(nf + 1, np.int32)
        ci = np.zeros(max(nnz, 1), np.int32)
        check(self._lib.pf_pattern(self._h, grid, rp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   ci.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))), "pf_pattern")
        return rp, ci[:nnz]

    def incidence(self, grid: int = 0, n_bus: int | None = None, n_branch: int | None = None):
        """(ptr, code, other) of grid `grid` in local numbering."""
        if n_bus is None or n_branch is None:
            if self.dims.n_grids != 1:
                raise ValueError("pass n_bus and n_branch for a multi-grid context")
            n_bus, n_branch = self.dims.n_bus, self.dims.n_branch
        ptr = np.zeros(n_bus + 1, np.int32)
        code = np.zeros(max(2 * n_branch, 1), np.int32)
        oth = np.zeros(max(2 * n_branch, 1), np.int32)
        ip = ctypes.POINTER(ctypes.c_int32)
        check(self._lib.pf_incidence(self._h, grid, ptr.ctypes.data_as(ip), code.ctypes.data_as(ip),
                                     oth.ctypes.data_as(ip)), "pf_incidence")
        return ptr, code[:2 * n_branch], oth[:2 * n_branch]

    def contributions(self, grid: int = 0):
        _, nnz, _ = self.grid_sizes(grid)
        ptr = np.zeros(nnz + 1, np.int64)
        check(self._lib.pf_contributions(self._h, grid, ptr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), None),
              "pf_contributions")
        src = np.zeros(max(int(ptr[-1]), 1), np.int32)
        check(self._lib.pf_contributions(self._h, grid, ptr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                         src.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))), "pf_contributions")
        return ptr, src[:int(ptr[-1])]

    # ---- buffers ----
    def empty_f(self, device=None):
        return torch.empty(self.dims.n_f, dtype=torch.float64, device=device or "cuda")

    def empty_vals(self, device=None):
        return torch.empty(self.dims.nnz, dtype=torch.float64, device=device or "cuda")

    # ---- evaluation ----
    def _overrides(self, p_inj=None, q_inj=None, status=None, br_r=None, br_x=None, br_b=None, br_tap=None,
                   gen_mode=None, gen_qlim=None):
        if all(v is None for v in (p_inj, q_inj, status, br_r, br_x, br_b, br_tap, gen_mode, gen_qlim)):
            return None
        d = self.dims
        ov = PfOverrides()
        ov.p_inj = _ptr(p_inj, numel=d.n_bus_inst, name="p_inj")
        ov.q_inj = _ptr(q_inj, numel=d.n_bus_inst, name="q_inj")
        ov.status = _ptr(status, torch.uint8, d.n_branch_inst, "status")
        ov.br_r = _ptr(br_r, numel=d.n_branch, name="br_r")
        ov.br_x = _ptr(br_x, numel=d.n_branch, name="br_x")
        ov.br_b = _ptr(br_b, numel=d.n_branch, name="br_b")
        ov.br_tap = _ptr(br_tap, numel=d.n_branch, name="br_tap")
        ov.gen_mode = _ptr(gen_mode, torch.uint8, d.n_gen_inst, "gen_mode")
        ov.gen_qlim = _ptr(gen_qlim, numel=d.n_gen_inst, name="gen_qlim")
        return ov

    def eval(self, x, F=None, vals=None, stream=None, **overrides):
        """Fused F and J (either output may be None to skip it)."""
        d = self.dims
        xp = _ptr(x, numel=d.n_x, name="x")
        fp = _ptr(F, numel=d.n_f, name="F")
        vp = _ptr(vals, numel=d.nnz, name="vals")
        ov = self._overrides(**overrides)
        check(self._lib.pf_eval(self._h, xp, ctypes.byref(ov) if ov is not None else None, fp, vp,
                                _stream(stream)), "pf_eval")
        return F, vals

    def eval_stage(self, stage: int, x, F=None, vals=None, stream=None, **overrides):
        """One kernel of an evaluation: stage 1 (phasors) or 2 (fused F/J; needs a preceding stage 1),
        with the per-call overrides of `eval`."""
        d = self.dims
        ov = self._overrides(**overrides)
        check(self._lib.pf_eval_stage(self._h, int(stage), _ptr(x, numel=d.n_x, name="x"),
                                      ctypes.byref(ov) if ov is not None else None,
                                      _ptr(F, numel=d.n_f, name="F"), _ptr(vals, numel=d.nnz, name="vals"),
                                      _stream(stream)), "pf_eval_stage")
        return F, vals

    def residual(self, x, F=None, stream=None):
        F = self.empty_f(x.device) if F is None else F
        check(self._lib.pf_residual(self._h, _ptr(x, numel=self.dims.n_x, name="x"),
                                    _ptr(F, numel=self.dims.n_f, name="F"), _stream(stream)), "pf_residual")
        return F

    def jacobian(self, x, vals=None, stream=None):
        vals = self.empty_vals(x.device) if vals is None else vals
        check(self._lib.pf_jacobian(self._h, _ptr(x, numel=self.dims.n_x, name="x"),
                                    _ptr(vals, numel=self.dims.nnz, name="vals"), _stream(stream)), "pf_jacobian")
        return vals

    def residual_jacobian(self, x, F=None, vals=None, stream=None):
        F = self.empty_f(x.device) if F is None else F
        vals = self.empty_vals(x.device) if vals is None else vals
        check(self._lib.pf_residual_jacobian(self._h, _ptr(x, numel=self.dims.n_x, name="x"),
                                             _ptr(F, numel=self.dims.n_f, name="F"),
                                             _ptr(vals, numel=self.dims.nnz, name="vals"), _stream(stream)),
              "pf_residual_jacobian")
        return F, vals

    def residual_jacobian_host(self, x: np.ndarray, F: np.ndarray | None, vals: np.ndarray | None, stream=None):
        """Host buffers in and out (float64, C-contiguous, ideally page-locked)."""
        def hp(a, n, name):
            if a is None:
                return None
            if a.dtype != np.float64 or not a.flags.c_contiguous or a.size != n:
                raise ValueError(f"{name}: float64 C-contiguous array of {n} elements required")
            return ctypes.c_void_p(a.ctypes.data)
        check(self._lib.pf_residual_jacobian_host(self._h, hp(x, self.dims.n_x, "x"), hp(F, self.dims.n_f, "F"),
                                                  hp(vals, self.dims.nnz, "vals"), _stream(stream)),
              "pf_residual_jacobian_host")

    def vjp(self, x, v, n_cot: int = 1, want=("x", "p_inj", "q_inj", "br_r", "br_x", "br_b", "br_tap"),
            stream=None, **overrides):
        """v: [n_cot * n_f] cotangents.  Returns a dict of [n_cot, ...] gradients."""
        d = self.dims
        xp = _ptr(x, numel=d.n_x, name="x")
        vp = _ptr(v, numel=n_cot * d.n_f, name="v")
        sizes = {"x": d.n_x, "p_inj": d.n_bus_inst, "q_inj": d.n_bus_inst, "br_r": d.n_branch_inst,
                 "br_x": d.n_branch_inst, "br_b": d.n_branch_inst, "br_tap": d.n_branch_inst}
        out = {k: torch.empty(n_cot, sizes[k], dtype=torch.float64, device=x.device) for k in want}
        g = PfGrads()
        for k, t in out.items():
            setattr(g, k, ctypes.c_void_p(t.data_ptr()))
        ov = self._overrides(**overrides)
        check(self._lib.pf_vjp(self._h, xp, ctypes.byref(ov) if ov is not None else None, vp, int(n_cot),
                               ctypes.byref(g), _stream(stream)), "pf_vjp")
        return out

    # ---- Newton iterations around the evaluation (tasks 3 and 4) ----
    def newton(self, x, tol: float = 1e-10, max_iter: int = 20, stream=None):
        """Newton power flow on every instance, x updated in place; returns
        {iterations, converged, max_mismatch, eval_ms, solve_ms, update_ms}."""
        info = PfNewtonInfo()
        check(self._lib.pf_newton(self._h, _ptr(x, numel=self.dims.n_x, name="x"), float(tol), int(max_iter),
                                  _stream(stream), ctypes.byref(info)), "pf_newton")
        return {k: getattr(info, k) for k, _ in PfNewtonInfo._fields_}

    def fdlf(self, x, tol: float = 1e-10, max_iter: int = 100, stream=None):
        """Fast decoupled power flow (reduced formulation), x updated in place."""
        info = PfNewtonInfo()
        check(self._lib.pf_fdlf(self._h, _ptr(x, numel=self.dims.n_x, name="x"), float(tol), int(max_iter),
                                _stream(stream), ctypes.byref(info)), "pf_fdlf")
        return {k: getattr(info, k) for k, _ in PfNewtonInfo._fields_}

    def set_newton_solver(self, solver: str = "lu"):
        """Linear solver of the Newton loop: "lu" (refactorization, default) or "qr"."""
        check(self._lib.pf_set_newton_solver(self._h, {"lu": 0, "qr": 1}[solver]), "pf_set_newton_solver")

    def newton_qlim(self, x, q_min, q_max, gen_mode=None, gen_qlim=None, tol: float = 1e-10, max_iter: int = 20,
                    max_rounds: int = 20, stream=None):
        """Extended-formulation Newton with reactive limits, x updated in place.
        gen_mode (uint8) / gen_qlim: starting modes (default all zero: voltage
        control), updated in place.  Returns (info dict, rounds, gen_mode, gen_qlim)."""
        d = self.dims
        if gen_mode is None:
            gen_mode = torch.zeros(d.n_gen_inst, dtype=torch.uint8, device=x.device)
        if gen_qlim is None:
            gen_qlim = torch.zeros(d.n_gen_inst, dtype=torch.float64, device=x.device)
        info = PfNewtonInfo()
        rounds = ctypes.c_int32(0)
        check(self._lib.pf_newton_qlim(self._h, _ptr(x, numel=d.n_x, name="x"), _ptr(q_min, numel=d.n_gen_inst,
                                       name="q_min"), _ptr(q_max, numel=d.n_gen_inst, name="q_max"),
                                       _ptr(gen_mode, torch.uint8, d.n_gen_inst, "gen_mode"),
                                       _ptr(gen_qlim, numel=d.n_gen_inst, name="gen_qlim"), float(tol),
                                       int(max_iter), int(max_rounds), _stream(stream), ctypes.byref(info),
                                       ctypes.byref(rounds)), "pf_newton_qlim")
        return {k: getattr(info, k) for k, _ in PfNewtonInfo._fields_}, rounds.value, gen_mode, gen_qlim

    def mismatch_norm(self, F, stream=None):
        """max |F| per instance ([n_inst] float64 CUDA tensor)."""
        out = torch.empty(self.dims.n_instances, dtype=torch.float64, device=F.device)
        check(self._lib.pf_mismatch_norm(self._h, _ptr(F, numel=self.dims.n_f, name="F"), _ptr(out),
                                         _stream(stream)), "pf_mismatch_norm")
        return out

    def newton_update(self, x, dx, stream=None):
        """x <- x - dx on the unknowns (dx in J's column order), in place."""
        check(self._lib.pf_newton_update(self._h, _ptr(x, numel=self.dims.n_x, name="x"),
                                         _ptr(dx, numel=self.dims.n_f, name="dx"), _stream(stream)),
              "pf_newton_update")
        return x

    # ---- tuning / errors ----
    @staticmethod
    def _tuning_dict(t):
        return {"tile_inc": t.tile_inc, "ctas_per_sm": t.ctas_per_sm, "split_rounds": t.split_rounds,
                "fuse_phasor": t.fuse_phasor}

    def tuning(self):
        t = PfTuning()
        check(self._lib.pf_get_tuning(self._h, ctypes.byref(t)), "pf_get_tuning")
        return self._tuning_dict(t)

    def set_tuning(self, tile_inc: int, ctas_per_sm: int = 0, split_rounds: int = 0, fuse_phasor: int = 0,
                   stream=None):
        t = PfTuning(int(tile_inc), int(ctas_per_sm), int(split_rounds), int(fuse_phasor))
        check(self._lib.pf_set_tuning(self._h, ctypes.byref(t), _stream(stream)), "pf_set_tuning")

    def autotune(self, x, F, vals, stream=None, cache=None):
        """Times the candidate tunings at x (F, vals: scratch outputs) and keeps the fastest.
        cache: path of a tuning file; an entry for this GPU and context shape is applied
        without timing ("from_cache" in the returned dict), else the choice is appended."""
        t = PfTuning()
        xp = _ptr(x, numel=self.dims.n_x, name="x")
        fp = _ptr(F, numel=self.dims.n_f, name="F")
        vp = _ptr(vals, numel=self.dims.nnz, name="vals")
        if cache is None:
            check(self._lib.pf_autotune(self._h, xp, fp, vp, _stream(stream), ctypes.byref(t)), "pf_autotune")
            return self._tuning_dict(t)
        hit = ctypes.c_int32(0)
        check(self._lib.pf_autotune_cache(self._h, os.fsencode(cache), xp, fp, vp, _stream(stream),
                                          ctypes.byref(t), ctypes.byref(hit)), "pf_autotune_cache")
        return dict(self._tuning_dict(t), from_cache=bool(hit.value))

    def sincos(self, theta, stream=None):
        """(cos, sin) of a float64 CUDA tensor by the evaluation's phasor routine."""
        n = theta.numel()
        c = torch.empty_like(theta)
        s = torch.empty_like(theta)
        check(self._lib.pf_sincos(self._h, _ptr(theta, numel=n, name="theta"), n, _ptr(c), _ptr(s),
                                  _stream(stream)), "pf_sincos")
        return c, s

    def voltage_records(self, x, stream=None):
        """[n_bus_inst, 4] float64 CUDA tensor of the evaluation's per-bus records
        (V cos theta, V sin theta, V, 1/V) at state x."""
        rec = torch.empty((self.dims.n_bus_inst, 4), dtype=torch.float64, device=x.device)
        check(self._lib.pf_voltage_records(self._h, _ptr(x, numel=self.dims.n_x, name="x"), _ptr(rec),
                                           _stream(stream)), "pf_voltage_records")
        return rec

    def check_device(self, stream=None):
        check(self._lib.pf_check_device(self._h, _stream(stream)), "pf_check_device")


def fp64_peak(device: int = 0, stream=None) -> tuple[float, float]:
    """The device's FP64 FMA rate (G operations/s) and the timed launch's
    duration (ms), measured by the library's pf_fp64_peak."""
    gops, ms = ctypes.c_double(), ctypes.c_double()
    with torch.cuda.device(device):
        check(_lib.load().pf_fp64_peak(int(device), ctypes.byref(gops), ctypes.byref(ms), _stream(stream)),
              "pf_fp64_peak")
    return gops.value, ms.value
