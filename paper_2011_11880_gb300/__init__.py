"""GB300-native power-flow residual and Jacobian evaluation.

Tasks (1) and (2) of Newton power flow (Sec. I of arXiv 2011.11880): bus
power-mismatch residuals F(theta, V) and the Jacobian values in a fixed
pattern, as sm_103a CUDA kernels behind the C ABI of include/pf.h
(libpf.so), with a batched multi-instance form and an adjoint
(vector-Jacobian product) behind torch.autograd.Function.

Importing this package loads libpf.so; if it has not been built the import
fails (there is no CPU fallback).
"""
from ._lib import PFError, load as _load

_load()

from .context import Context, Dims, fp64_peak  # noqa: E402
from .autograd import PFResidual, residual  # noqa: E402

__all__ = ["Context", "Dims", "PFError", "PFResidual", "fp64_peak", "residual"]
