"""Seeded synthetic workloads of the split-step path (inputs only; none of the method's arithmetic).

The paper measures on synthetic turbulence only, so every workload here is a parameter set plus
seeds; the random numbers the method itself draws (screen noise) come from Philox inside the path.
Seeds follow seed = 0x2604072480 + config id.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 0x2604072480
LAMBDA = 1.55e-6
L0_INNER = 5e-3
L0_OUTER = 10.0


@dataclass
class Workload:
    name: str
    N: int
    dx: float
    L: float
    S: int
    cn2: list
    w0: list                 # source waists [m]; <= 0 means plane wave
    sh_levels: int = 0
    alpha: float = 0.0
    time_steps: int = 1
    realizations: int = 1
    seed: int = SEED_BASE
    extra: dict = field(default_factory=dict)

    @property
    def dz(self):
        return [self.L / self.S] * self.S


def config1(vacuum: bool = False) -> Workload:
    """Plain split-step, one realization: N = 128, dx = 2 mm, L = 1 km, 5 screens, Cn^2 = 1e-15
    (or 0 for the vacuum run), Gaussian w0 = 2 cm, no subharmonics."""
    return Workload("split-step N=128 S=5 (1 realization)", 128, 2e-3, 1000.0, 5, [0.0 if vacuum else 1e-15] * 5,
                    [0.02], seed=SEED_BASE + 1)


def config2_cn2() -> list:
    """8 log-spaced Cn^2 values from 1e-16 to 1e-13: 10^(-16 + 3 i / 7)."""
    return [10.0 ** (-16.0 + 3.0 * i / 7.0) for i in range(8)]


def config2(cn2: float) -> Workload:
    """Monte Carlo: N = 512, dx = 1 mm, L = 2 km, 10 screens, 3-level subharmonics, plane wave and
    Gaussian w0 = 2 cm sharing each realization's screens, 1000 realizations per Cn^2."""
    return Workload(f"monte-carlo N=512 S=10 SH Cn2={cn2:.3g}", 512, 1e-3, 2000.0, 10, [cn2] * 10, [0.0, 0.02],
                    sh_levels=3, realizations=1000, seed=SEED_BASE + 2)


def config3() -> Workload:
    """Temporal evolution: N = 1024, dx = 0.5 mm, L = 1 km, 16 screens, Cn^2 = 1e-15, AR alpha = 0.99,
    256 time steps, 8 Gaussian beams w0 = 1.0 + 0.25 b cm sharing each step's screens."""
    return Workload("ar-evolution N=1024 S=16 B=8 T=256", 1024, 5e-4, 1000.0, 16, [1e-15] * 16,
                    [0.01 + 0.0025 * b for b in range(8)], alpha=0.99, time_steps=256, seed=SEED_BASE + 3)


def config4_instances(n: int = 64, seed: int = SEED_BASE + 4):
    """Uneven batch: n instances with N from {256, 512, 1024, 2048}, S uniform in 4..20 and
    log10 Cn^2 uniform in [-16, -14] (numpy PCG64 stream of the seed)."""
    rng = np.random.default_rng(seed)
    Ns = rng.choice([256, 512, 1024, 2048], size=n)
    Ss = rng.integers(4, 21, size=n)
    cn2 = 10.0 ** rng.uniform(-16.0, -14.0, size=n)
    return [dict(N=int(a), S=int(b), cn2=float(c), dx=2e-3, L=1000.0, w0=0.02) for a, b, c in zip(Ns, Ss, cn2)]


def config5() -> Workload:
    """Differentiable path: N = 512, dx = 1 mm, L = 1 km, 10 screens, Cn^2 = 5e-16, Gaussian w0 = 2 cm,
    batch 64; two 512 x 512 phase masks initialised to seeded N(0, 0.1 rad)."""
    return Workload("d2nn N=512 S=10 B=64", 512, 1e-3, 1000.0, 10, [5e-16] * 10, [0.02], realizations=64,
                    seed=SEED_BASE + 5, extra=dict(aperture=0.3048))


def config5_masks(N: int = 512, seed: int = SEED_BASE + 5):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, 0.1, (N, N)).astype(np.float32), rng.normal(0.0, 0.1, (N, N)).astype(np.float32)
