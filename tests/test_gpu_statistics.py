"""Monte Carlo statistics on the GPU path against theory (Sec. 3.2-3.3): plane-wave scintillation
index in weak turbulence from 400 realizations accumulated with the on-device FP64 Welford merge,
and the second-moment radius of a Gaussian beam in vacuum."""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2604_07248_gb300 as ts  # noqa: E402

LAM = 1.55e-6
K = 2 * np.pi / LAM
DEV = torch.device("cuda:0")


def test_plane_wave_scintillation_matches_first_order_rytov():
    # N = 512, dx = 1 mm, L = 2 km in 10 screens, Cn^2 = 7e-16 (sigma_R^2 ~ 0.05), pure Kolmogorov
    # spectrum without subharmonics (periodic screens keep the periodic grid seamless).
    N, dx, L, S, cn2, R, chunk = 512, 1e-3, 2000.0, 10, 7e-16, 400, 100
    dz = L / S
    plan = ts.Plan(LAM, N, dx, [dz] * S, [cn2] * S, l0=0.0, L0=np.inf, max_batch=chunk)
    plan.set_sources([0.0])  # plane wave
    U = torch.zeros((chunk, N, N), dtype=torch.complex64, device=DEV)
    I = torch.zeros((chunk, N, N), dtype=torch.float32, device=DEV)
    mean = torch.zeros((1, N, N), dtype=torch.float64, device=DEV)
    m2 = torch.zeros_like(mean)
    count = 0
    for c in range(R // chunk):
        plan.propagate(U, chunk, flags=ts.TS_PROP_SOURCE | ts.TS_PROP_INTENSITY | ts.TS_PROP_NO_FIELD,
                       seed=0x2604072482, real_base=c * chunk, intensity=I)
        plan.moments_accumulate(I, chunk, 1, count, mean, m2)
        count += chunk
    si_mean = torch.zeros(1, dtype=torch.float64, device=DEV)
    plan.moments_finalize(mean, m2, 1, count, si_mean=si_mean)
    torch.cuda.synchronize()
    si = si_mean.item()
    assert abs(mean.mean().item() - 1.0) < 1e-3  # energy of a unit plane wave is conserved
    md = O.medium(LAM, N, dx, l0=0.0, L0=np.inf)
    amp2 = O.psd_amplitude(md, cn2, dz) ** 2
    f = np.fft.fftfreq(N, 1 / N) * 2 * np.pi / (N * dx)
    k2 = f[None, :] ** 2 + f[:, None] ** 2
    z = [L - s * dz for s in range(1, S + 1)]
    grid = sum(4 * np.sum(amp2 * np.sin(k2 * zs / (2 * K)) ** 2) for zs in z)
    cont = 2.25 * K ** (7 / 6) * cn2 * dz * sum(zs ** (5 / 6) for zs in z)
    assert abs(grid / cont - 1) < 0.05
    assert abs(si / grid - 1) < 0.08, (si, grid)


def test_vacuum_second_moment_radius_is_the_beam_radius():
    # Gaussian w0 = 2 cm over 2 km in vacuum: W(L) = w0 sqrt(1 + (L / zR)^2), and the second-moment
    # radius sqrt(2 sum r^2 I / sum I) of a Gaussian equals W (S23).
    N, dx, L, S, w0 = 512, 1e-3, 2000.0, 10, 0.02
    plan = ts.Plan(LAM, N, dx, [L / S] * S, [0.0] * S, max_batch=2)
    plan.set_sources([w0])
    U = torch.zeros((2, N, N), dtype=torch.complex64, device=DEV)
    I = torch.zeros((2, N, N), dtype=torch.float32, device=DEV)
    sums = torch.zeros((2, 2), dtype=torch.float64, device=DEV)
    plan.propagate(U, 2, flags=ts.TS_PROP_SOURCE | ts.TS_PROP_INTENSITY, intensity=I, beam_sums=sums)
    # the same radius through the boundary's moment calls (one group, two realizations)
    mean = torch.zeros((1, N, N), dtype=torch.float64, device=DEV)
    m2 = torch.zeros_like(mean)
    acc = torch.zeros((1, 2), dtype=torch.float64, device=DEV)
    w_lt = torch.zeros(1, dtype=torch.float64, device=DEV)
    plan.moments_accumulate(I, 2, 1, 0, mean, m2, beam_sums=sums, beam_acc=acc)
    plan.moments_finalize(mean, m2, 1, 2, beam_acc=acc, w_lt=w_lt)
    torch.cuda.synchronize()
    zR = np.pi * w0 ** 2 / LAM
    W = w0 * np.sqrt(1 + (L / zR) ** 2)
    wlt = np.sqrt(2 * sums[0, 1].item() / sums[0, 0].item())
    assert abs(wlt / W - 1) < 1e-4
    assert abs(w_lt[0].item() / W - 1) < 1e-4
