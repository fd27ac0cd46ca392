"""The Monte Carlo workload (Sec. 3.2-3.3) against theory over its whole Cn^2 sweep.

N = 512, dx = 1 mm, L = 2 km in 10 screens (propagate, then screen), l0 = 5 mm, L0 = 10 m, eight
Cn^2 values 10^(-16 + 3 i / 7) (sigma_R^2 from 0.007 to 7.1), 1000 realizations per value, plane
wave and a 2 cm Gaussian through the same screens, moments accumulated in FP64 on the device.

Theory, evaluated for the discrete model from the oracle's FP64 amplitudes:
  * plane-wave scintillation, first-order Rytov for thin screens: a screen at distance d before the
    receiver contributes 4 sum_kappa s(kappa)^2 sin^2(kappa^2 d / 2k) (weak fluctuations);
  * long-term radius of the Gaussian beam (S23 / S24 as second moments): a phase screen adds its
    mean-square gradient / k^2 to the beam's mean-square angle, so in expectation
    W_LT^2 = W(L)^2 + 2 sum_s (d_s / k)^2 sum_kappa |kappa|^2 s_s(kappa)^2 (subharmonic cells
    included), exact for the paraxial equation at any strength until light wraps around the grid.
The subharmonic screens of the configuration are not periodic, so a plane wave on the periodic
grid picks up scintillation from their seam; the plane-wave Rytov check therefore runs without
subharmonics, and the configured screens (with subharmonics) are checked through the Gaussian beam,
which stays clear of the grid edge.
"""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2604_07248_gb300 as ts  # noqa: E402
from paper_2604_07248_gb300 import workloads as W  # noqa: E402

DEV = torch.device("cuda:0")
K = 2 * np.pi / W.LAMBDA


def run_sweep_point(cn2, sh, R=1000, chunk=50):
    """(mean intensity of the plane wave, plane-wave SI over the grid, Gaussian on-axis SI,
    Gaussian W_LT) from R realizations through the library."""
    wl = W.config2(cn2)
    N, S = wl.N, wl.S
    B = 2 * chunk
    plan = ts.Plan(W.LAMBDA, N, wl.dx, wl.dz, [cn2] * S, l0=W.L0_INNER, L0=W.L0_OUTER, sh_levels=sh, max_batch=B)
    plan.set_sources([0.0, 0.02])  # field 2r: plane wave, 2r + 1: Gaussian, both through screens r
    ph = torch.zeros((chunk, S, N, N), dtype=torch.complex64, device=DEV)
    U = torch.zeros((B, N, N), dtype=torch.complex64, device=DEV)
    I = torch.zeros((B, N, N), dtype=torch.float32, device=DEV)
    sums = torch.zeros((B, 2), dtype=torch.float64, device=DEV)
    mean = torch.zeros((2, N, N), dtype=torch.float64, device=DEV)
    m2 = torch.zeros_like(mean)
    acc = torch.zeros((2, 2), dtype=torch.float64, device=DEV)
    count = 0
    i = W.config2_cn2().index(cn2)
    for c in range(R // chunk):
        plan.make_screens(None, wl.seed, real_base=i * 1000 + c * chunk, n_real=chunk, phasor=ph)
        plan.propagate(U, B, phasor=ph, phi_group=2,
                       flags=ts.TS_PROP_SOURCE | ts.TS_PROP_INTENSITY | ts.TS_PROP_NO_FIELD, intensity=I, beam_sums=sums)
        plan.moments_accumulate(I, B, 2, count, mean, m2, beam_sums=sums, beam_acc=acc)
        count += chunk
    si_mean = torch.zeros(2, dtype=torch.float64, device=DEV)
    si_c = torch.zeros(2, dtype=torch.float64, device=DEV)
    w_lt = torch.zeros(2, dtype=torch.float64, device=DEV)
    plan.moments_finalize(mean, m2, 2, count, si_mean=si_mean, si_center=si_c, beam_acc=acc, w_lt=w_lt)
    torch.cuda.synchronize()
    out = (float(mean[0].mean().item()), float(si_mean[0].item()), float(si_c[1].item()), float(w_lt[1].item()))
    plan.close()
    return out


def theory(cn2, sh):
    """(continuous sigma_R^2, discrete-screen plane-wave Rytov SI, moment-theorem W_LT of the beam)."""
    wl = W.config2(cn2)
    N, dx, L, S = wl.N, wl.dx, wl.L, wl.S
    dz = L / S
    md = O.medium(W.LAMBDA, N, dx, l0=W.L0_INNER, L0=W.L0_OUTER)
    s2 = O.psd_amplitude(md, cn2, dz) ** 2
    f = np.fft.fftfreq(N, 1 / N) * 2 * np.pi / (N * dx)
    k2 = f[None, :] ** 2 + f[:, None] ** 2
    d = [L - s * dz for s in range(1, S + 1)]
    rytov = sum(4 * np.sum(s2 * np.sin(k2 * ds / (2 * K)) ** 2) for ds in d)
    grad2 = np.sum(k2 * s2)
    if sh:
        b = O.sh_amplitude(md, cn2, dz)
        dk = 2 * np.pi / (N * dx)
        for p in range(1, 4):
            for q in range(9):
                kx, ky = (q % 3 - 1) * dk / 3 ** p, (q // 3 - 1) * dk / 3 ** p
                grad2 += (kx * kx + ky * ky) * b[p - 1, q] ** 2
    zR = np.pi * 0.02 ** 2 / W.LAMBDA
    Wv = 0.02 * np.sqrt(1 + (L / zR) ** 2)
    w_mom = np.sqrt(Wv ** 2 + 2 * sum((ds / K) ** 2 for ds in d) * grad2)
    sig_r2 = 1.23 * cn2 * K ** (7 / 6) * L ** (11 / 6)
    return sig_r2, rytov, w_mom


def test_config2_sweep_against_rytov_and_the_moment_theorem():
    for cn2 in W.config2_cn2():
        sig_r2, rytov, _ = theory(cn2, 0)
        m_pl, si_pl, si_g0, _ = run_sweep_point(cn2, 0)
        _, _, w_mom = theory(cn2, 3)
        m_pl3, _, si_g3, w_lt3 = run_sweep_point(cn2, 3)
        # energy of a unit plane wave is conserved (|H| = |exp(i phi)| = 1)
        assert abs(m_pl - 1) < 1e-3 and abs(m_pl3 - 1) < 1e-3
        if sig_r2 < 0.5:
            # weak fluctuations: the plane-wave SI is the discrete-screen Rytov sum (1000 realizations
            # over the whole grid: a few per cent of statistical spread)
            assert abs(si_pl / rytov - 1) < 0.05, (cn2, si_pl, rytov)
        else:
            # saturation (Sec. 3.3): below first-order theory
            assert si_pl < rytov
        # the configured screens (with subharmonics): long-term radius of the Gaussian beam
        tol = 0.02 if sig_r2 < 0.5 else 0.08  # strong turbulence: wide-angle light wraps around the grid
        assert abs(w_lt3 / w_mom - 1) < tol, (cn2, w_lt3, w_mom)
        if sig_r2 < 0.2:
            # the subharmonics (large-scale tilt and curvature) leave the beam's on-axis SI unchanged in
            # weak turbulence; the grid noise is the same with and without them
            assert abs(si_g3 / si_g0 - 1) < 0.05, (cn2, si_g3, si_g0)
