"""torch.autograd.Function over the library's residual and adjoint kernels.

Forward evaluates F(x; P_inj, Q_inj, r, x, b_c, tau) with pf_eval; backward
runs pf_vjp, which recomputes the trigonometric terms instead of keeping any
forward intermediates.  A batch of cotangents is expressed the autograd way:
pass the state (and any parameter) expanded along a leading axis of length B
with stride 0 (``x.expand(B, -1)``); the output is then [B, n_f] and one
backward call evaluates all B vector-Jacobian products with a single kernel
launch, returning [B, ...] gradients.
"""
from __future__ import annotations

import torch

from .context import Context

_PARAMS = ("p_inj", "q_inj", "br_r", "br_x", "br_b", "br_tap")


def _base(t, n, name):
    """(1-D base tensor, B or None) of a [n] tensor or a stride-0 [B, n] expansion."""
    if t is None:
        return None, None
    if t.dim() == 1:
        if t.shape[0] != n:
            raise ValueError(f"{name}: expected {n} entries")
        return t.contiguous(), None
    if t.dim() == 2 and t.shape[1] == n and (t.stride(0) == 0 or t.shape[0] == 1):
        return t[0].contiguous(), t.shape[0]
    raise ValueError(f"{name}: expected shape [{n}] or a stride-0 expansion [B, {n}] of one vector")


class PFResidual(torch.autograd.Function):
    """F = PFResidual.apply(ctx, x, p_inj, q_inj, br_r, br_x, br_b, br_tap).

    Parameters may be None (the values built into ``ctx`` are used).  In the
    batched-cotangent form every tensor argument that is not None must be the
    same stride-0 [B, .] expansion length B.
    """

    @staticmethod
    def forward(fctx, pfctx: Context, x, p_inj=None, q_inj=None, br_r=None, br_x=None, br_b=None, br_tap=None):
        d = pfctx.dims
        sizes = {"p_inj": d.n_bus_inst, "q_inj": d.n_bus_inst, "br_r": d.n_branch, "br_x": d.n_branch,
                 "br_b": d.n_branch, "br_tap": d.n_branch}
        x0, B = _base(x, d.n_x, "x")
        bases, batched = {}, {}
        for name, t in zip(_PARAMS, (p_inj, q_inj, br_r, br_x, br_b, br_tap)):
            bases[name], b = _base(t, sizes[name], name)
            batched[name] = b is not None
            if b is not None and b != B:
                raise ValueError(f"{name}: batch length {b} differs from x's {B}")
        if B is not None and any(t is not None and not batched[n] for n, t in bases.items()):
            raise ValueError("with a batched x, parameters must be expanded to the same batch length")
        F = torch.empty(d.n_f, dtype=torch.float64, device=x0.device)
        pfctx.eval(x0, F, None, **bases)
        fctx.pfctx = pfctx
        fctx.B = B
        fctx.given = {n: bases[n] is not None for n in _PARAMS}
        fctx.save_for_backward(x0, *[bases[n] for n in _PARAMS])
        return F if B is None else F.unsqueeze(0).expand(B, d.n_f)

    @staticmethod
    def backward(fctx, gF):
        pfctx: Context = fctx.pfctx
        x0, *pb = fctx.saved_tensors
        bases = dict(zip(_PARAMS, pb))
        B = fctx.B
        n_cot = 1 if B is None else B
        v = gF.contiguous().reshape(-1)
        want = ["x"] + [n for n in _PARAMS if fctx.needs_input_grad[2 + _PARAMS.index(n)]]
        want = list(dict.fromkeys(want))
        g = pfctx.vjp(x0, v, n_cot=n_cot, want=want, **bases)

        def shape(t):
            return t[0] if B is None else t

        out = [None, shape(g["x"]) if fctx.needs_input_grad[1] else None]
        for n in _PARAMS:
            out.append(shape(g[n]) if n in g and fctx.needs_input_grad[2 + _PARAMS.index(n)] else None)
        return tuple(out)


def residual(pfctx: Context, x, p_inj=None, q_inj=None, br_r=None, br_x=None, br_b=None, br_tap=None):
    """Differentiable residual F(x, ...) (see PFResidual)."""
    return PFResidual.apply(pfctx, x, p_inj, q_inj, br_r, br_x, br_b, br_tap)
