"""D2NN training loop of Sec. 2.5 on the library's calls (one turbulence realization per epoch).

Per epoch: the source beam propagates through a fresh realization of the path's screens (regenerated
from the seed, realization index = epoch), the two-mask receiver forms the intensity and its MAE loss
against the apertured free-space intensity, the receiver adjoint gives the mask gradients, and one
Adam step per mask follows, with the learning rate of a one-cycle schedule.  The masks start at a
constant phase (zero), as the paper states.  Only the masks train, so no adjoint propagation runs.
"""
from __future__ import annotations

import math

import numpy as np

from . import binding as bd


def one_cycle_lr(step: int, total: int, lr_max: float, pct_start: float = 0.3, div_factor: float = 25.0,
                 final_div_factor: float = 1e4) -> float:
    """One-cycle learning rate (Smith & Topin 2019) with cosine annealing: from lr_max / div_factor up
    to lr_max over the first pct_start of the steps, then down to lr_max / div_factor / final_div_factor
    at the last step (step counted from 0)."""
    lr0 = lr_max / div_factor
    lr_end = lr0 / final_div_factor
    up_end = float(pct_start * total) - 1.0
    if step <= up_end:
        frac, a, b = (step / up_end if up_end > 0 else 1.0), lr0, lr_max
    else:
        span = (total - 1) - up_end
        frac, a, b = ((step - up_end) / span if span > 0 else 1.0), lr_max, lr_end
    return b + (a - b) * 0.5 * (1.0 + math.cos(math.pi * min(max(frac, 0.0), 1.0)))


def hv57_path(lam: float, L: float, sigma_r2: float, N: int, dx: float, rytov_limit: float, V: float = 21.0,
              samples: int = 1501, max_screens: int = 64):
    """A vertical Hufnagel-Valley path of length L whose ground constant A gives the whole path the
    Rytov variance sigma_r2 (S19 is linear in A, so two evaluations fix it), and its screen placement
    (Sec. 2.4).  Returns (A, heights, Cn^2 samples, dz[], Cn^2[] per interval)."""
    h = np.linspace(0.0, L, samples)
    base = bd.rytov_interval(h, bd.cn2_hufnagel_valley(h, V, 0.0), lam, 0.0, L)
    unit = bd.rytov_interval(h, bd.cn2_hufnagel_valley(h, V, 1.0) - bd.cn2_hufnagel_valley(h, V, 0.0), lam, 0.0, L)
    A = (sigma_r2 - base) / unit
    if not A > 0:
        raise ValueError("the requested Rytov variance is below the profile's A-independent part")
    cn2 = bd.cn2_hufnagel_valley(h, V, A)
    dz, cn, _ = bd.place_screens(h, cn2, lam, N, dx, L, rytov_limit, max_screens=max_screens)
    return A, h, cn2, dz, cn


class D2nnTrainer:
    """Holds the plan, the reference intensity, the masks and their Adam states on one device."""

    def __init__(self, lam, N, dx, dz, cn2, w0, aperture, seed, epochs, lr_max=0.01, l0=0.0, L0=0.0, device=None,
                 loss_kind=0, init_masks=None):
        import torch

        self.torch = torch
        dev = device or torch.device("cuda", torch.cuda.current_device())
        self.plan = bd.Plan(lam, N, dx, dz, cn2, l0=l0, L0=L0, max_batch=1)
        self.plan.set_sources([w0])
        vac = bd.Plan(lam, N, dx, dz, [0.0] * len(dz), max_batch=1)
        vac.set_sources([w0])
        U = torch.zeros((1, N, N), dtype=torch.complex64, device=dev)
        vac.propagate(U, 1, flags=bd.TS_PROP_SOURCE)
        z = torch.zeros((N, N), dtype=torch.float32, device=dev)
        I = torch.zeros((1, N, N), dtype=torch.float32, device=dev)
        vac.d2nn_forward(U, 1, z, z, aperture, z, 1, torch.zeros((3, 1, N, N), dtype=torch.complex64, device=dev), I,
                         torch.zeros(1, dtype=torch.float64, device=dev))
        vac.close()
        self.Iref = I[0].clone()  # its own storage: self.I below is overwritten every epoch
        # intensities normalised to the free-space peak: the loss (and gradient) scale 1 / peak for the
        # MAE, 1 / peak^2 for the squared error
        peak = float(self.Iref.max().item())
        self.loss_scale = 1.0 / peak if loss_kind == 0 else 1.0 / (peak * peak)
        self.plan.set_loss_scale(self.loss_scale)
        if init_masks is None:  # constant initial phase, as in the paper
            self.th = [torch.zeros((N, N), dtype=torch.float32, device=dev) for _ in range(2)]
        else:
            self.th = [torch.as_tensor(np.asarray(mk, np.float32)).to(dev) for mk in init_masks]
        self.m = [torch.zeros_like(z) for _ in range(2)]
        self.v = [torch.zeros_like(z) for _ in range(2)]
        self.g = [torch.zeros_like(z) for _ in range(2)]
        self.U = U
        self.I = I
        self.ws = torch.zeros((3, 1, N, N), dtype=torch.complex64, device=dev)
        self.gU = torch.zeros_like(U)
        self.loss = torch.zeros(1, dtype=torch.float64, device=dev)
        self.aperture, self.seed, self.epochs, self.lr_max = aperture, seed, epochs, lr_max
        self.loss_kind = loss_kind  # 0 = mean |I - Iref| (the paper's MAE), 1 = mean squared error
        self.t = 0

    def epoch(self, e: int, stream=None):
        """One epoch on realization e (asynchronous; the loss stays on the device in self.loss)."""
        p = self.plan
        p.propagate(self.U, 1, flags=bd.TS_PROP_SOURCE, seed=self.seed, real_base=e, stream=stream)
        p.d2nn_forward(self.U, 1, self.th[0], self.th[1], self.aperture, self.Iref, self.loss_kind, self.ws, self.I,
                       self.loss, stream=stream)
        p.d2nn_backward(1, self.th[0], self.th[1], self.aperture, self.Iref, self.loss_kind, self.ws, self.I,
                        self.g[0], self.g[1], self.gU, stream=stream)
        self.t += 1
        lr = one_cycle_lr(e, self.epochs, self.lr_max)
        for k in range(2):
            bd.adam_step(self.th[k], self.g[k], self.m[k], self.v[k], self.t, lr, stream=stream)
