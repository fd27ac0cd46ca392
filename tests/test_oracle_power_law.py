"""Pins for the oracle's power-law media (Table S1, S11-S15), CPU only: the PSD constant against its
defining integral, the Kolmogorov special case, the phase structure function of a pure power law in
closed form, and PSD recovery / structure function of the synthesised screens."""
import math

import numpy as np
import pytest
from scipy import integrate, special

import oracle as O

LAM = 1.55e-6
K = 2 * np.pi / LAM


def _index_sf_integral(alpha):
    """int_0^inf (1 - sin u / u) u^(2 - alpha) du, numerically (3 < alpha < 5)."""
    # below eps the integrand is u^(4 - alpha) / 6 (1 - u^2 / 20 + ...): integrated in closed form
    eps = 1e-3
    head = eps ** (5 - alpha) / (6 * (5 - alpha)) * (1 - 3 * (5 - alpha) / (20 * (7 - alpha)) * eps ** 2)
    head += integrate.quad(lambda u: (1 - np.sinc(u / np.pi)) * u ** (2 - alpha), eps, 1, limit=200)[0]
    # tail: int_1^inf u^(2-alpha) du - int_1^inf sin(u) u^(1-alpha) du
    tail = 1 / (alpha - 3) - integrate.quad(lambda u: u ** (1 - alpha), 1, np.inf, weight="sin", wvar=1)[0]
    return head + tail


@pytest.mark.parametrize("alpha", [3.2, 11 / 3, 4.0, 4.3, 4.8])
def test_power_law_constant_gives_unit_structure_constant(alpha):
    # D_n(r) = 8 pi int (1 - sin(kappa r)/(kappa r)) A Cn^2 kappa^-alpha kappa^2 dkappa = Cn^2 r^(alpha-3)
    # exactly when 8 pi A I(alpha) = 1, for the structure-constant reading of Cn^2
    A = O.power_law_constant(alpha)
    assert abs(8 * np.pi * A * _index_sf_integral(alpha) - 1) < 1e-6


def test_power_law_constant_at_kolmogorov_is_0033():
    assert abs(O.power_law_constant(11 / 3) / 0.033 - 1) < 2e-4


def test_default_medium_is_the_kolmogorov_power_law():
    md = O.medium(LAM, 64, 1e-3, l0=5e-3, L0=10.0)
    mk = O.medium(LAM, 64, 1e-3, l0=5e-3, L0=10.0, alpha=11 / 3, A=0.033)
    assert np.array_equal(O.psd_amplitude(md, 1e-14, 100.0), O.psd_amplitude(mk, 1e-14, 100.0))
    assert np.array_equal(O.sh_amplitude(md, 1e-14, 100.0), O.sh_amplitude(mk, 1e-14, 100.0))


@pytest.mark.parametrize("alpha", [3.2, 4.3])
def test_phase_psd_power_law_scaling(alpha):
    A = O.power_law_constant(alpha)
    md = O.medium(LAM, 64, 1e-3, l0=0.0, L0=np.inf, alpha=alpha, A=A)
    cn2, dz = 1e-15, 10.0
    for kap in (5.0, 77.0):
        # S15: Phi_phi = 2 pi k^2 dz A Cn^2 kappa^-alpha; doubling kappa scales by 2^-alpha
        assert abs(O.phase_psd(md, cn2, dz, kap ** 2) / (2 * np.pi * K ** 2 * dz * A * cn2 * kap ** -alpha) - 1) < 1e-12
        assert abs(O.phase_psd(md, cn2, dz, 4 * kap ** 2) / O.phase_psd(md, cn2, dz, kap ** 2) - 2 ** -alpha) < 1e-12


def _phase_sf_closed_form(alpha):
    """int_0^inf (1 - J0(u)) u^(1 - alpha) du = pi / (2^mu Gamma((mu+1)/2)^2 sin(pi (mu-1)/2)),
    mu = alpha - 1 (2 < alpha < 4)."""
    mu = alpha - 1
    return np.pi / (2 ** mu * special.gamma((mu + 1) / 2) ** 2 * np.sin(np.pi * (mu - 1) / 2))


@pytest.mark.parametrize("alpha", [3.2, 11 / 3, 3.8])
def test_phase_structure_function_closed_form(alpha):
    # D_phi(r) = 2 int Phi_phi (1 - J0(kappa r)) d^2 kappa = 4 pi c r^(alpha-2) int (1 - J0(u)) u^(1-alpha) du
    # for Phi_phi = c kappa^-alpha; the closed form reduces to 6.88 (r/r0)^(5/3) at alpha = 11/3
    A = O.power_law_constant(alpha)
    md = O.medium(LAM, 64, 1e-3, l0=0.0, L0=np.inf, alpha=alpha, A=A)
    cn2, dz = 1e-15, 100.0
    c = 2 * np.pi * K ** 2 * dz * A * cn2
    for r in (0.01, 0.2):
        f = lambda u: 2 * O.phase_psd(md, cn2, dz, (u / r) ** 2) * (1 - special.j0(u)) * 2 * np.pi * (u / r) / r
        val = sum(integrate.quad(f, a, b, limit=400)[0] for a, b in [(0, 1), (1, 10), (10, 100), (100, np.inf)])
        closed = 4 * np.pi * c * r ** (alpha - 2) * _phase_sf_closed_form(alpha)
        assert abs(val / closed - 1) < 0.01, (alpha, r, val / closed)
    if abs(alpha - 11 / 3) < 1e-12:
        r0 = (0.423 * K ** 2 * cn2 * dz) ** (-3 / 5)
        closed = 4 * np.pi * (2 * np.pi * K ** 2 * dz * 0.033 * cn2) * _phase_sf_closed_form(alpha)
        assert abs(closed / (6.88 * r0 ** (-5 / 3)) - 1) < 0.002


def test_psd_recovery_biological_tissue():
    # Table S1 biological tissue, alpha = 4.3, with an outer scale: averaging |FFT2(phi)|^2 / N^4 over
    # screens recovers s(kappa)^2 for every kappa off the DC and Nyquist lines
    N, M, alpha = 64, 600, 4.3
    md = O.medium(LAM, N, 2e-3, l0=5e-3, L0=0.5, alpha=alpha, A=O.power_law_constant(alpha))
    cn2, dz = 1e-14, 200.0
    amp2 = O.psd_amplitude(md, cn2, dz) ** 2
    acc = np.zeros((N, N))
    for s in range(M):
        acc += np.abs(np.fft.fft2(O.make_screen(md, cn2, dz, 0, 78, s, 0))) ** 2 / N ** 4
    acc /= M
    f = np.fft.fftfreq(N, 1 / N)
    FX, FY = np.meshgrid(f, f)
    ok = (FX != 0) & (FY != 0) & (np.abs(FX) != N / 2) & (np.abs(FY) != N / 2)
    rad = np.sqrt(FX ** 2 + FY ** 2)
    for lo, hi in [(1, 2), (2, 4), (4, 8), (8, 16), (16, 31)]:
        sel = ok & (rad >= lo) & (rad < hi)
        ratio = np.mean(acc[sel] / amp2[sel])
        assert abs(ratio - 1) < 4 / np.sqrt(M * sel.sum()) + 1e-3, (lo, hi, ratio)


def test_power_law_screens_follow_the_closed_form_structure_function():
    # alpha = 3.4 (a non-Kolmogorov atmosphere, Table S1), 3-level subharmonics, l0 = 0, L0 = inf: the
    # sample structure function of the screens follows D_phi(r) = 4 pi c I(alpha) r^(alpha - 2) at
    # separations well inside the grid
    N, dx, cn2, dz, M, alpha = 128, 4e-3, 1e-14, 100.0, 150, 3.4
    A = O.power_law_constant(alpha)
    md = O.medium(LAM, N, dx, l0=0.0, L0=np.inf, alpha=alpha, A=A)
    lags = (2, 8)
    D = np.zeros(len(lags))
    for s in range(M):
        phi = O.make_screen(md, cn2, dz, 3, 101, s, 0)
        for i, lag in enumerate(lags):
            D[i] += 0.5 * (np.mean((phi[:, lag:] - phi[:, :-lag]) ** 2) + np.mean((phi[lag:] - phi[:-lag]) ** 2))
    D /= M
    c = 2 * np.pi * K ** 2 * dz * A * cn2
    for i, lag in enumerate(lags):
        th = 4 * np.pi * c * (lag * dx) ** (alpha - 2) * _phase_sf_closed_form(alpha)
        assert abs(D[i] / th - 1) < 0.2, (lag, D[i] / th)
    # log-log slope between the two lags close to alpha - 2
    slope = math.log(D[1] / D[0]) / math.log(lags[1] / lags[0])
    assert abs(slope - (alpha - 2)) < 0.15, slope
