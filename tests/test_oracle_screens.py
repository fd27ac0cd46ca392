"""Pins for the oracle's phase screens (CPU only): PSD constants, PSD recovery, structure function,
subharmonics and AR(1) evolution, each against a closed form or an exact expectation."""
import numpy as np
import pytest
from scipy import integrate, special

import oracle as O

LAM = 1.55e-6
K = 2 * np.pi / LAM


def r0_of(cn2, dz):
    """Fried parameter of one interval, S18."""
    return (0.423 * K ** 2 * cn2 * dz) ** (-3 / 5)


def test_phase_psd_integrates_to_kolmogorov_structure_function():
    # D(r) = 2 int Phi_phi(kappa) (1 - J0(kappa r)) d^2kappa must equal 6.88 (r/r0)^(5/3) for the
    # pure power law (l0 = 0, L0 = inf): ties 2 pi * 0.033 (S14, S17) to 0.423 (S18).
    md = O.medium(LAM, 64, 1e-3, l0=0.0, L0=np.inf)
    cn2, dz = 1e-15, 100.0
    r0 = r0_of(cn2, dz)
    for r in (0.01, 0.05, 0.3):
        f = lambda u: 2 * O.phase_psd(md, cn2, dz, (u / r) ** 2) * (1 - special.j0(u)) * 2 * np.pi * (u / r) / r
        val = sum(integrate.quad(f, a, b, limit=400)[0] for a, b in [(0, 1), (1, 10), (10, 100), (100, np.inf)])
        assert abs(val / (6.88 * (r / r0) ** (5 / 3)) - 1) < 0.01


def test_phase_psd_matches_s17_in_cycles_per_metre():
    # S17 in spatial frequency f = kappa / 2 pi with measure d^2 f: 0.023 r0^(-5/3) f^(-11/3).
    md = O.medium(LAM, 64, 1e-3, l0=0.0, L0=np.inf)
    cn2, dz = 3e-15, 50.0
    r0 = r0_of(cn2, dz)
    for kap in (1.0, 30.0, 900.0):
        f = kap / (2 * np.pi)
        s17 = 0.023 * r0 ** (-5 / 3) * f ** (-11 / 3) / (2 * np.pi) ** 2
        assert abs(O.phase_psd(md, cn2, dz, kap ** 2) / s17 - 1) < 0.01


def test_psd_shape_scales():
    md = O.medium(LAM, 64, 1e-3, l0=0.0, L0=np.inf)
    # pure power law: Phi(2 kappa) / Phi(kappa) = 2^(-11/3); linear in Cn^2 and dz (S14)
    for kap in (5.0, 77.0):
        assert abs(O.phase_psd(md, 1e-15, 10, 4 * kap ** 2) / O.phase_psd(md, 1e-15, 10, kap ** 2) - 2 ** (-11 / 3)) < 1e-12
    assert abs(O.phase_psd(md, 2e-15, 30, 9.0) / O.phase_psd(md, 1e-15, 10, 9.0) - 6) < 1e-12
    # outer scale flattens the spectrum at kappa << kappa0; inner scale rolls it off as exp(-kappa^2/kappa_m^2)
    mo = O.medium(LAM, 64, 1e-3, l0=0.0, L0=10.0)
    assert abs(O.phase_psd(mo, 1e-15, 1, 1e-8) / O.phase_psd(mo, 1e-15, 1, 0.0) - 1) < 1e-6
    mi = O.medium(LAM, 64, 1e-3, l0=5e-3, L0=np.inf)
    km = 2 * np.pi / 5e-3
    assert abs(O.phase_psd(mi, 1e-15, 1, km ** 2) / O.phase_psd(md, 1e-15, 1, km ** 2) - np.exp(-1)) < 1e-12


def test_psd_recovery_expectation():
    # Sec. 3.1: averaging |FFT2(phi)|^2 / N^4 over screens recovers s(kappa)^2 (exactly, in expectation,
    # for every kappa off the DC and Nyquist lines).
    N, M = 64, 1000
    md = O.medium(LAM, N, 2e-3, l0=5e-3, L0=10.0)
    cn2, dz = 1e-14, 200.0
    amp2 = O.psd_amplitude(md, cn2, dz) ** 2
    acc = np.zeros((N, N))
    for s in range(M):
        acc += np.abs(np.fft.fft2(O.make_screen(md, cn2, dz, 0, 77, s, 0))) ** 2 / N ** 4
    acc /= M
    f = np.fft.fftfreq(N, 1 / N)
    FX, FY = np.meshgrid(f, f)
    ok = (FX != 0) & (FY != 0) & (np.abs(FX) != N / 2) & (np.abs(FY) != N / 2)
    rad = np.sqrt(FX ** 2 + FY ** 2)
    for lo, hi in [(1, 2), (2, 4), (4, 8), (8, 16), (16, 31)]:
        sel = ok & (rad >= lo) & (rad < hi)
        ratio = np.mean(acc[sel] / amp2[sel])
        assert abs(ratio - 1) < 4 / np.sqrt(M * sel.sum()) + 1e-3, (lo, hi, ratio)


def _exact_structure_function(md, cn2, dz, sh, lag):
    """E[(phi(x + r) - phi(x))^2] of the discrete model: sum 2 s^2 (1 - cos(kappa . r)) over the grid
    and the subharmonic cells, averaged over the x and y directions."""
    N, dx = md.N, md.dx
    s = O.psd_amplitude(md, cn2, dz)
    dk = 2 * np.pi / (N * dx)
    f = np.fft.fftfreq(N, 1 / N) * dk
    KX, KY = np.meshgrid(f, f)
    r = lag * dx
    D = 0.5 * (np.sum(2 * s ** 2 * (1 - np.cos(KX * r))) + np.sum(2 * s ** 2 * (1 - np.cos(KY * r))))
    if sh:
        b = O.sh_amplitude(md, cn2, dz)
        for p in range(1, 4):
            for q in range(9):
                mp, nq = q // 3 - 1, q % 3 - 1
                kx, ky = nq * dk / 3 ** p, mp * dk / 3 ** p
                D += 0.5 * (2 * b[p - 1, q] ** 2 * (2 - np.cos(kx * r) - np.cos(ky * r)))
    return D


@pytest.mark.parametrize("sh", [0, 3])
def test_screen_structure_function_matches_model(sh):
    N, dx, cn2, dz, M = 128, 4e-3, 1e-14, 100.0, 150
    md = O.medium(LAM, N, dx, l0=0.0, L0=np.inf)
    lags = (1, 4, 16, 48)
    D = np.zeros(len(lags))
    for s in range(M):
        phi = O.make_screen(md, cn2, dz, sh, 99, s, 0)
        for i, lag in enumerate(lags):
            D[i] += 0.5 * (np.mean((phi[:, lag:] - phi[:, :-lag]) ** 2) + np.mean((phi[lag:] - phi[:-lag]) ** 2))
    D /= M
    for i, lag in enumerate(lags):
        ex = _exact_structure_function(md, cn2, dz, sh, lag)
        assert abs(D[i] / ex - 1) < 0.08, (lag, D[i] / ex)


def _ring_integral(md, cn2, dz, h, ni, mi):
    """Integral of the phase PSD over the cell [ni - 1/2, ni + 1/2] x [mi - 1/2, mi + 1/2] (units of h),
    by adaptive 2-D quadrature of phase_psd alone."""
    f = lambda ky, kx: O.phase_psd(md, cn2, dz, kx * kx + ky * ky)
    return integrate.dblquad(f, (ni - 0.5) * h, (ni + 0.5) * h, (mi - 0.5) * h, (mi + 0.5) * h,
                             epsabs=0, epsrel=1e-9)[0]


def test_subharmonic_amplitudes_carry_the_psd_of_their_cells():
    # Two-sided pin of the subharmonic amplitudes (Eq. 2): cell (n', m') of level p stands for the
    # square of side dk / 3^p centred on (n', m') dk / 3^p, so its variance b^2 must be the phase PSD
    # integrated over that cell.  With an outer scale much smaller than the grid (kappa0 = 2 pi / L0
    # well above dk) the PSD is smooth across every subharmonic cell and the midpoint value times the
    # cell area equals the integral to O((cell / kappa0)^2): a factor 3^p or sqrt(3) in any level's
    # amplitude, or a frequency at the wrong scale, is off by far more than the tolerance.
    N, dx, cn2, dz = 64, 2e-3, 1e-14, 100.0
    md = O.medium(LAM, N, dx, l0=0.0, L0=0.02)
    dk = 2 * np.pi / (N * dx)
    b = O.sh_amplitude(md, cn2, dz)
    for p in range(1, 4):
        h = dk / 3 ** p
        assert b[p - 1, 4] == 0.0
        for q in range(9):
            mi, ni = q // 3 - 1, q % 3 - 1
            if mi == 0 and ni == 0:
                continue
            ratio = b[p - 1, q] ** 2 / _ring_integral(md, cn2, dz, h, ni, mi)
            assert abs(ratio - 1) < 2e-3 * 9.0 ** (1 - p) + 1e-5, (p, q, ratio)


def test_subharmonic_levels_replicate_the_first_grid_ring():
    # For the pure power law (l0 = 0, L0 = inf) the PSD is self-similar, so each subharmonic level is a
    # 1/3^p scale copy of the FFT grid's first ring of 8 bins around DC: the fraction of the ring's PSD
    # integral that the 8 point samples carry is the same number for the grid (amplitudes from
    # psd_amplitude, pinned by the PSD-recovery expectation) and for every level.  The number itself
    # (about 0.60: point samples under-weight the kappa^(-11/3) rise toward the origin) is the known
    # low-frequency deficit of the method; a wrong 3^p scaling of an amplitude changes it by 9^p.
    N, dx, cn2, dz = 64, 2e-3, 1e-14, 100.0
    md = O.medium(LAM, N, dx, l0=0.0, L0=np.inf)
    dk = 2 * np.pi / (N * dx)
    s = O.psd_amplitude(md, cn2, dz)
    ring = [(ni, mi) for mi in (-1, 0, 1) for ni in (-1, 0, 1) if (ni, mi) != (0, 0)]
    grid = sum(s[mi % N, ni % N] ** 2 for ni, mi in ring) / sum(_ring_integral(md, cn2, dz, dk, ni, mi) for ni, mi in ring)
    assert 0.55 < grid < 0.65
    b = O.sh_amplitude(md, cn2, dz)
    for p in range(1, 4):
        h = dk / 3 ** p
        lev = sum(b[p - 1, q] ** 2 for q in range(9)) / sum(_ring_integral(md, cn2, dz, h, ni, mi) for ni, mi in ring)
        assert abs(lev / grid - 1) < 1e-6, (p, lev, grid)


def test_subharmonic_screens_have_the_structure_function_of_their_coefficients():
    # The subharmonic part of an oracle screen (same seed with and without subharmonics: the grid noise
    # is drawn from its own counters) is a sum of 24 random plane waves, so its expected structure
    # function is sum_q 2 b_q^2 (1 - cos(kappa_q . r)) (Re and Im of the noise each N(0,1)).  The Monte
    # Carlo average over the screens' pixels must reach it: pins the noise normalisation and the
    # frequencies (n', m') dk / 3^p that the screen synthesis places the amplitudes at.
    N, dx, cn2, dz, M = 32, 2e-3, 1e-14, 100.0, 2000
    md = O.medium(LAM, N, dx, l0=0.0, L0=np.inf)
    dk = 2 * np.pi / (N * dx)
    lags = (2, 8, 31)
    vals = np.zeros((M, len(lags)))
    for sidx in range(M):
        d = O.make_screen(md, cn2, dz, 3, 11, sidx, 0) - O.make_screen(md, cn2, dz, 0, 11, sidx, 0)
        for i, lag in enumerate(lags):
            vals[sidx, i] = 0.5 * (np.mean((d[:, lag:] - d[:, :-lag]) ** 2) + np.mean((d[lag:] - d[:-lag]) ** 2))
    b = O.sh_amplitude(md, cn2, dz)
    for i, lag in enumerate(lags):
        r = lag * dx
        ex = 0.0
        for p in range(1, 4):
            for q in range(9):
                kx, ky = (q % 3 - 1) * dk / 3 ** p, (q // 3 - 1) * dk / 3 ** p
                ex += b[p - 1, q] ** 2 * (2 - np.cos(kx * r) - np.cos(ky * r))
        mc, se = vals[:, i].mean(), vals[:, i].std() / np.sqrt(M)
        assert abs(mc - ex) < 5 * se, (lag, mc / ex, se / ex)


def test_kolmogorov_structure_function_with_subharmonics():
    # Kolmogorov structure function (Eq. 2-3, S18): l0 = 0, L0 = inf, N = 256, 3-level subharmonics.  (1) The oracle's
    # screens reach the exact expectation of the discrete model at every lag.  (2) Against
    # 6.88 (r / r0)^(5/3) for 2 dx <= r <= N dx / 8 the model lies between 0.75 and 0.95: the grid
    # square itself holds >= 0.98 of D(r) (polar quadrature below), and the remaining deficit is the
    # point sampling of the kappa^(-11/3) spectrum in the cells bordering the origin (each level carries
    # 0.60 of its ring's PSD, the test above), which grows toward large r (0.89 at r = 2 dx, 0.77 at
    # N dx / 8 for this grid).  (3) Without subharmonics the large-r deficit is more than twice as deep.
    N, dx, cn2, dz, M = 256, 2e-3, 1e-14, 100.0, 240
    md = O.medium(LAM, N, dx, l0=0.0, L0=np.inf)
    r0 = r0_of(cn2, dz)
    lags = (2, 4, 8, 16, 32)
    vals = np.zeros((M, len(lags)))
    for sidx in range(M):
        phi = O.make_screen(md, cn2, dz, 3, 2604, sidx, 0)
        for i, lag in enumerate(lags):
            vals[sidx, i] = 0.5 * (np.mean((phi[:, lag:] - phi[:, :-lag]) ** 2) + np.mean((phi[lag:] - phi[:-lag]) ** 2))
    K = np.pi / dx
    for i, lag in enumerate(lags):
        r = lag * dx
        th = 6.88 * (r / r0) ** (5 / 3)
        model = _exact_structure_function(md, cn2, dz, 3, lag)
        mc, se = vals[:, i].mean(), vals[:, i].std() / np.sqrt(M)
        assert abs(mc - model) < 5 * se, (lag, mc / model, se / model)
        assert 0.75 < model / th < 0.95, (lag, model / th)
        if lag in (2, 32):
            # fraction of D(r) inside the grid square |kx|, |ky| < pi / dx, in polar coordinates
            def wedge(t):
                g = lambda k: 2 * O.phase_psd(md, cn2, dz, k * k) * (
                    1 - 0.5 * (np.cos(k * np.cos(t) * r) + np.cos(k * np.sin(t) * r))) * k
                pts = [0.0, 1 / r, 10 / r, K / np.cos(t)]
                return sum(integrate.quad(g, a, c, limit=400)[0] for a, c in zip(pts[:-1], pts[1:]))
            inside = 8 * integrate.quad(wedge, 0, np.pi / 4, limit=100)[0]
            assert 0.98 < inside / th < 1.01, (lag, inside / th)
    big = _exact_structure_function(md, cn2, dz, 0, 32) / (6.88 * (32 * dx / r0) ** (5 / 3))
    assert big < 0.5 and 1 - big > 2 * (1 - _exact_structure_function(md, cn2, dz, 3, 32) / (6.88 * (32 * dx / r0) ** (5 / 3)))


def test_subharmonic_screen_separable_form():
    # Eq. 2 evaluated as a rank-3-per-level separable product equals the term-by-term sum.
    N, dx = 32, 3e-3
    md = O.medium(LAM, N, dx, l0=0.0, L0=np.inf)
    rng = np.random.default_rng(1)
    a = rng.standard_normal((3, 9)) + 1j * rng.standard_normal((3, 9))
    a[:, 4] = 0
    direct = O.sh_screen(md, a)
    dk = 2 * np.pi / (N * dx)
    x = np.arange(N) * dx
    sep = np.zeros((N, N))
    for p in range(1, 4):
        dkp = dk / 3 ** p
        ex = np.exp(1j * np.outer([-1, 0, 1], x) * dkp)  # [n'][i]
        ey = np.exp(1j * np.outer([-1, 0, 1], x) * dkp)  # [m'][j]
        A = a[p - 1].reshape(3, 3)  # [m'][n']
        sep += np.real(ey.T @ A @ ex)
    assert np.max(np.abs(direct - sep)) < 1e-12 * np.abs(direct).max()


def test_screen_mean_is_removed():
    md = O.medium(LAM, 64, 2e-3, l0=5e-3, L0=10.0)
    for sh in (0, 3):
        phi = O.make_screen(md, 1e-13, 200.0, sh, 5, 0, 0)
        assert abs(phi.mean()) < 1e-13 * np.abs(phi).max()


def test_ar_preserves_spectral_variance_and_correlates_as_alpha_power():
    # Eq. 5: E|spec_t|^2 = 2 s^2 for every t (the sqrt(1 - alpha^2) weight) and
    # E[spec_0 conj(spec_t)] = alpha^t 2 s^2, bin by bin.  The screens' ensemble correlation follows
    # alpha^tau too and crosses the 0.4 threshold of Fig. 3C near tau = ln 0.4 / ln alpha.
    N, alpha, T, R = 32, 0.9, 24, 24
    md = O.medium(LAM, N, 2e-3, l0=5e-3, L0=0.05)
    cn2, dz = 1e-14, 100.0
    amp2 = O.psd_amplitude(md, cn2, dz) ** 2
    nz = amp2 > 0
    var_ratio, spec_corr = np.zeros(T), np.zeros(T)
    cov, v0, vt = np.zeros(T), np.zeros(T), np.zeros(T)
    for r in range(R):
        spec, sh = O.screen_spectrum(md, cn2, dz, 3, 42, 0, r, 0)
        spec0 = spec.copy()
        phi0 = O.screen_from_spectrum(md, spec, sh)
        for t in range(1, T + 1):
            spec, sh = O.ar_step(md, cn2, dz, 3, 42, 0, r, t, alpha, spec, sh)
            var_ratio[t - 1] += np.mean(np.abs(spec[nz]) ** 2 / (2 * amp2[nz])) / R
            spec_corr[t - 1] += np.mean(np.real(spec0[nz] * np.conj(spec[nz])) / (2 * amp2[nz])) / R
            phi = O.screen_from_spectrum(md, spec, sh)
            cov[t - 1] += np.sum(phi0 * phi)
            v0[t - 1] += np.sum(phi0 ** 2)
            vt[t - 1] += np.sum(phi ** 2)
    tau = np.arange(1, T + 1)
    n = R * nz.sum()
    assert np.all(np.abs(var_ratio - 1) < 5 * np.sqrt(2.0 / n) + 0.01)
    assert np.all(np.abs(spec_corr - alpha ** tau) < 5 / np.sqrt(n))
    corr = cov / np.sqrt(v0 * vt)
    assert np.max(np.abs(corr - alpha ** tau)) < 0.1
    crossing = np.log(0.4) / np.log(alpha)
    assert np.all(corr[tau < crossing - 3] > 0.4) and np.all(corr[tau > crossing + 3] < 0.4)


def test_ar_translation_is_an_exact_shift():
    # Eq. 4 with alpha = 1: multiplying by exp(-2 pi i T f.v) shifts the screen by v T.
    N, dx = 32, 2e-3
    md = O.medium(LAM, N, dx, l0=5e-3, L0=10.0)
    spec, _ = O.screen_spectrum(md, 1e-14, 100.0, 0, 3, 0, 0, 0)
    phi0 = O.screen_from_spectrum(md, spec)
    T, vx, vy = 0.01, 3 * dx / 0.01, -2 * dx / 0.01
    spec1, _ = O.ar_step(md, 1e-14, 100.0, 0, 3, 0, 0, 1, 1.0, spec, None, vx=vx, vy=vy, T=T)
    phi1 = O.screen_from_spectrum(md, spec1)
    assert np.max(np.abs(phi1 - np.roll(phi0, (-2, 3), axis=(0, 1)))) < 1e-10 * np.abs(phi0).max()
