"""Oracle for path planning (TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``).

Plain numpy restatements, written independently of the CUDA library's host code:

* ``hv_cn2``: the Hufnagel-Valley profile, S21, written out;
* ``rytov_interval``: S19 by composite Simpson quadrature of the piecewise-linear profile (the library
  integrates the linear pieces in closed form instead);
* ``place_screens``: the placement routine of Sec. 2.4 in the order the paper lists its steps, with
  the readings stated in the repository's design notes: midpoint splits, greedy merges, a final sweep
  that extends each interval to the Rytov limit (lengths found here by plain bisection), kept when it
  needs no more intervals, then equal splits of intervals longer than the Eq. 7 limit.

Pinned by ``tests/test_oracle_planner.py``: S19 reduces to 1.226 k^(7/6) Cn^2 L^(11/6) for a constant
profile (the plane-wave Rytov variance), HV5/7 gives r0 = 5 cm and theta0 = 7 urad at 0.5 um (its
name), and constant-profile placements have the closed-form interval length.
"""
from __future__ import annotations

import numpy as np


def hv_cn2(h, V=21.0, A=1.7e-14):
    """Hufnagel-Valley Cn^2(h) (S21)."""
    h = np.asarray(h, dtype=np.float64)
    return (0.00594 * (V / 27.0) ** 2 * (1e-5 * h) ** 10 * np.exp(-h / 1000.0)
            + 2.7e-16 * np.exp(-h / 1500.0) + A * np.exp(-h / 100.0))


def _interp(prof_z, prof_cn2, z):
    # linear between samples, constant beyond the ends (np.interp's convention)
    return np.interp(z, prof_z, prof_cn2)


def rytov_interval(prof_z, prof_cn2, lam, z0, z1, n=40001):
    """sigma_R^2 = 3.27 k^(7/6) dz^(5/6) int_0^dz Cn2(z0 + z) (1 - z/dz)^(5/3) dz  (S19), Simpson's rule."""
    dz = z1 - z0
    if dz <= 0:
        return 0.0
    k = 2 * np.pi / lam
    z = np.linspace(0.0, dz, n)
    f = _interp(prof_z, prof_cn2, z0 + z) * (1.0 - z / dz) ** (5.0 / 3.0)
    h = dz / (n - 1)
    integral = h / 3.0 * (f[0] + f[-1] + 4.0 * f[1:-1:2].sum() + 2.0 * f[2:-1:2].sum())
    return 3.27 * k ** (7.0 / 6.0) * dz ** (5.0 / 6.0) * integral


def path_integral(prof_z, prof_cn2, z0, z1, n=40001):
    """int_{z0}^{z1} Cn2(z) dz (trapezoid on a fine grid)."""
    z = np.linspace(z0, z1, n)
    f = _interp(prof_z, prof_cn2, z)
    return float((z[1] - z[0]) * (f.sum() - 0.5 * (f[0] + f[-1])))


def max_step(lam, N, dx, n0=1.0):
    """Eq. 7 as read in this repository: dz_max = (N dx / 2) sqrt(k^2 - kmax^2) / kmax, kmax = pi / dx."""
    k = 2 * np.pi * n0 / lam
    kmax = np.pi / dx
    return 0.5 * N * dx * np.sqrt(k * k - kmax * kmax) / kmax


def place_screens(prof_z, prof_cn2, lam, N, dx, L, rytov_limit, init_bounds=(), n0=1.0):
    """Sec. 2.4 placement; returns (dz, cn2_eff, rytov) numpy arrays."""
    lam_eff = lam / n0
    ry = lambda a, b: rytov_interval(prof_z, prof_cn2, lam_eff, a, b)  # noqa: E731
    # 1. the caller's intervals
    b = [0.0] + [x for x in sorted(init_bounds) if 0.0 < x < L] + [L]
    b = [x for i, x in enumerate(b) if i == 0 or x > b[i - 1]]
    # 2. midpoint splits above the limit
    i = 0
    while i + 1 < len(b):
        if ry(b[i], b[i + 1]) > rytov_limit and b[i + 1] - b[i] > 1e-6 * L:
            b.insert(i + 1, 0.5 * (b[i] + b[i + 1]))
        else:
            i += 1
    # 3. greedy merges while the merged interval stays within the limit
    i = 0
    while i + 2 < len(b):
        if ry(b[i], b[i + 2]) <= rytov_limit:
            del b[i + 1]
        else:
            i += 1
    # 4. sweep: each interval extended until its variance reaches the limit (bisection)
    f = [0.0]
    while f[-1] < L * (1 - 1e-12):
        z0 = f[-1]
        if ry(z0, L) <= rytov_limit:
            f.append(L)
            break
        lo, hi = 0.0, L - z0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if ry(z0, z0 + mid) < rytov_limit:
                lo = mid
            else:
                hi = mid
            if hi - lo <= 1e-10 * (1.0 + hi):
                break
        f.append(min(L, z0 + max(lo, 1e-9 * L)))
    f[-1] = L
    best = f if len(f) <= len(b) else b
    # 5. equal splits of intervals longer than the Eq. 7 limit
    dzm = max_step(lam, N, dx, n0)
    out = [0.0]
    for a, c in zip(best[:-1], best[1:]):
        parts = max(1, int(np.ceil((c - a) / dzm * (1 - 1e-12))))
        out += [a + (c - a) * j / parts for j in range(1, parts + 1)]
    out = np.asarray(out)
    dz = np.diff(out)
    cn2 = np.array([path_integral(prof_z, prof_cn2, a, c) / (c - a) for a, c in zip(out[:-1], out[1:])])
    ryt = np.array([ry(a, c) for a, c in zip(out[:-1], out[1:])])
    return dz, cn2, ryt
