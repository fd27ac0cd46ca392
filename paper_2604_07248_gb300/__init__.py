"""GB300-native split-step optical-turbulence path (TurPy, arXiv 2604.07248).

The compute lives in the CUDA library ``libturbscreen.so`` (``csrc/``, C ABI in
``include/turbscreen.h``); this package holds its ctypes binding and a torch.autograd.Function
around the propagate/adjoint pair.  PyTorch supplies device memory and streams only.
"""
from __future__ import annotations

from .binding import (TS_BATCH_NO_TUNE, TS_BATCH_TEST_STALL, TS_PLAN_ALLOW_ALIASING, TS_PLAN_SPLIT_BF16, TS_PLAN_TEST_STALL, TS_PROP_INTENSITY,
                      TS_PROP_NO_FIELD, TS_PROP_SOURCE, Batch, Plan, TsError, cn2_hufnagel_valley, load, max_step,
                      philox4x32_10, place_screens, power_law_constant, rytov_interval)

__all__ = ["Plan", "Batch", "TsError", "TS_BATCH_NO_TUNE", "TS_BATCH_TEST_STALL", "load", "max_step", "philox4x32_10", "propagate",
           "cn2_hufnagel_valley", "rytov_interval", "place_screens", "power_law_constant", "TS_PROP_SOURCE",
           "TS_PROP_INTENSITY", "TS_PROP_NO_FIELD", "TS_PLAN_ALLOW_ALIASING", "TS_PLAN_SPLIT_BF16",
           "TS_PLAN_TEST_STALL"]


def _autograd():
    import torch

    class SplitStep(torch.autograd.Function):
        """U_out = P(U_in) (Eq. 1 over the plan's S steps); backward applies the hand-written
        adjoint P^H (conj H, exp(-i phi), reversed order), regenerating the screens from their seed
        when no screen tensor is given."""

        @staticmethod
        def forward(ctx, field, plan, phi, phi_group, seed, real_base):
            out = field.detach().resolve_conj().contiguous().clone()
            B = out.shape[0] if out.dim() == 3 else 1
            plan.propagate(out, B, phi=phi, phi_group=phi_group, seed=seed, real_base=real_base)
            ctx.plan, ctx.phi, ctx.meta = plan, phi, (B, phi_group, seed, real_base)
            return out

        @staticmethod
        def backward(ctx, grad):
            B, phi_group, seed, real_base = ctx.meta
            g = grad.detach().resolve_conj().contiguous().clone()
            ctx.plan.propagate_backward(g, B, phi=ctx.phi, phi_group=phi_group, seed=seed, real_base=real_base)
            return g, None, None, None, None, None

    return SplitStep


_SPLIT = None


def propagate(field, plan: Plan, phi=None, phi_group: int = 1, seed: int = 0, real_base: int = 0):
    """Differentiable split-step propagation of complex64 fields [B, N, N] on the plan's device."""
    global _SPLIT
    if _SPLIT is None:
        _SPLIT = _autograd()
    return _SPLIT.apply(field, plan, phi, phi_group, seed, real_base)
