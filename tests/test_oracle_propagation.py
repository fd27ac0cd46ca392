"""Pins for the oracle's propagation, moments and D2NN receiver (CPU only): analytic Gaussian beam,
energy conservation, adjoint identities, Rytov scintillation, Welford moments, finite differences."""
import numpy as np
import pytest

import oracle as O

LAM = 1.55e-6
K = 2 * np.pi / LAM


def gaussian_beam(N, dx, w0, z):
    """Paraxial Gaussian beam without its exp(i k z) piston: (w0/W) exp(-r^2/W^2) exp(i k r^2 / 2R) exp(-i psi)."""
    zR = np.pi * w0 ** 2 / LAM
    W = w0 * np.sqrt(1 + (z / zR) ** 2)
    R = z * (1 + (zR / z) ** 2)
    psi = np.arctan(z / zR)
    x = (np.arange(N) - N // 2) * dx
    r2 = x[None, :] ** 2 + x[:, None] ** 2
    return (w0 / W) * np.exp(-r2 / W ** 2) * np.exp(1j * K * r2 / (2 * R)) * np.exp(-1j * psi), W


def rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_vacuum_gaussian_matches_analytic_beam():
    # 128-point grid, dx = 2 mm, w0 = 2 cm, L = 1 km in five 200 m steps, Cn^2 = 0 (vacuum run).
    N, dx, w0, L, S = 128, 2e-3, 0.02, 1000.0, 5
    md = O.medium(LAM, N, dx)
    U = O.propagate(md, [L / S] * S, None, O.source_gaussian(N, dx, w0))
    ref, W = gaussian_beam(N, dx, w0, L)
    assert abs(W - 0.03176) < 1e-4
    assert rel_l2(U, ref) < 1e-6
    # the second-moment radius sqrt(2 sum r^2 I / sum I) of a Gaussian beam is W(L) (Sec. 3.2, S23)
    sI, sR = O.beam_sums(N, dx, np.abs(U) ** 2)
    assert abs(np.sqrt(2 * sR / sI) / W - 1) < 1e-5


def test_transfer_function_properties():
    md = O.medium(LAM, 64, 1e-3)
    H = O.transfer(md, 150.0)
    assert np.max(np.abs(np.abs(H) - 1)) < 1e-14
    assert np.max(np.abs(O.transfer(md, 0.0) - 1)) == 0.0
    # composition: H(a) H(b) = H(a + b)
    assert np.max(np.abs(O.transfer(md, 40.0) * O.transfer(md, 110.0) - H)) < 1e-12
    # small-kappa expansion of the phase: -dz (kappa^2 / 2k + kappa^4 / 8k^3 + ...)
    dk = 2 * np.pi / (64 * 1e-3)
    assert abs(np.angle(H[0, 1]) + 150.0 * (dk ** 2 / (2 * K) + dk ** 4 / (8 * K ** 3))) < 1e-14


def test_energy_is_conserved_through_turbulence():
    N, dx = 64, 2e-3
    md = O.medium(LAM, N, dx, l0=5e-3, L0=10.0)
    phi = np.stack([O.make_screen(md, 1e-13, 100.0, 3, 9, s, 0) for s in range(4)])
    U0 = O.source_gaussian(N, dx, 0.02)
    U = O.propagate(md, [100.0] * 4, phi, U0)
    assert abs(np.sum(np.abs(U) ** 2) / np.sum(np.abs(U0) ** 2) - 1) < 1e-12


def test_propagation_adjoint_identities():
    # <P x, y> = <x, P^H y> and P^H P = I (P is unitary: |H| = |exp(i phi)| = 1).
    N, dx = 32, 2e-3
    md = O.medium(LAM, N, dx, l0=5e-3, L0=10.0)
    phi = np.stack([O.make_screen(md, 1e-13, 50.0, 0, 2, s, 0) for s in range(3)])
    rng = np.random.default_rng(0)
    x = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    y = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    dz = [30.0, 50.0, 70.0]
    Px = O.propagate(md, dz, phi, x)
    PHy = O.propagate_adjoint(md, dz, phi, y)
    assert abs(np.vdot(y, Px) - np.vdot(PHy, x)) < 1e-12 * np.linalg.norm(x) * np.linalg.norm(y)
    assert rel_l2(O.propagate_adjoint(md, dz, phi, Px), x) < 1e-13


def test_propagation_gradient_matches_finite_differences():
    # L = sum |P(U)|^4 w; gradient wrt Re/Im of U by central differences equals P^H applied to dL/dU'.
    N, dx = 16, 3e-3
    md = O.medium(LAM, N, dx, l0=5e-3, L0=10.0)
    phi = np.stack([O.make_screen(md, 1e-12, 50.0, 0, 4, s, 0) for s in range(2)])
    rng = np.random.default_rng(2)
    U = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    w = rng.random((N, N))
    dz = [50.0, 50.0]

    def loss(u):
        v = O.propagate(md, dz, phi, u)
        return np.sum(w * np.abs(v) ** 4)

    V = O.propagate(md, dz, phi, U)
    g = O.propagate_adjoint(md, dz, phi, 4 * w * np.abs(V) ** 2 * V)
    eps = 1e-6
    for (j, i) in [(0, 0), (3, 7), (15, 15), (8, 2)]:
        e = np.zeros((N, N))
        e[j, i] = eps
        d_re = (loss(U + e) - loss(U - e)) / (2 * eps)
        d_im = (loss(U + 1j * e) - loss(U - 1j * e)) / (2 * eps)
        assert abs(d_re - g[j, i].real) < 1e-6 * abs(g).max()
        assert abs(d_im - g[j, i].imag) < 1e-6 * abs(g).max()


def test_weak_turbulence_plane_wave_scintillation_rytov():
    # Sec. 3.3 / S26 in the weak regime.  Plane wave, 2 km path, 5 screens without subharmonics (a
    # periodic screen keeps the periodic grid seamless).  First-order (Rytov) theory for thin screens:
    #   SI = 4 sum_s sum_kappa s_s(kappa)^2 sin^2(kappa^2 z_s / 2k)            (on the grid)
    #      -> 2.25 k^(7/6) Cn^2 dz sum_s z_s^(5/6)                            (continuum)
    #      -> 1.23 Cn^2 k^(7/6) L^(11/6) = sigma_R^2                           (continuous path)
    N, dx, L, S, cn2, M = 256, 2e-3, 2000.0, 5, 2e-15, 40
    dz = L / S
    md = O.medium(LAM, N, dx, l0=0.0, L0=np.inf)
    W = O.Welford((N, N))
    for r in range(M):
        phi = np.stack([O.make_screen(md, cn2, dz, 0, 1234, s, r) for s in range(S)])
        W.update(np.abs(O.propagate(md, [dz] * S, phi, np.ones((N, N), complex))) ** 2)
    si = W.si_map().mean()
    amp2 = O.psd_amplitude(md, cn2, dz) ** 2
    f = np.fft.fftfreq(N, 1 / N) * 2 * np.pi / (N * dx)
    k2 = f[None, :] ** 2 + f[:, None] ** 2
    z = [L - s * dz for s in range(1, S + 1)]
    grid = sum(4 * np.sum(amp2 * np.sin(k2 * zs / (2 * K)) ** 2) for zs in z)
    cont = 2.25 * K ** (7 / 6) * cn2 * dz * sum(zs ** (5 / 6) for zs in z)
    sigma_r2 = 1.23 * cn2 * K ** (7 / 6) * L ** (11 / 6)
    assert abs(grid / cont - 1) < 0.03
    assert abs(si / grid - 1) < 0.12
    # discrete screens undershoot the continuous path by the quadrature of the 5 screens
    assert 0.7 < si / sigma_r2 < 0.95


def test_welford_matches_population_variance_and_merge():
    rng = np.random.default_rng(5)
    x = rng.gamma(2.0, 3.0, size=(50, 8, 8)) + 1e6  # large offset: Welford must not cancel
    W = O.Welford((8, 8))
    for a in x:
        W.update(a)
    assert np.max(np.abs(W.M2 / W.n - x.var(axis=0))) < 1e-6
    assert np.max(np.abs(W.mean - x.mean(axis=0))) < 1e-8
    A, B = O.Welford((8, 8)), O.Welford((8, 8))
    for a in x[:17]:
        A.update(a)
    for a in x[17:]:
        B.update(a)
    A.merge(B)
    assert A.n == 50
    assert np.max(np.abs(A.M2 - W.M2)) < 1e-6 * W.M2.max()
    assert np.max(np.abs(A.mean - W.mean)) < 1e-9


def test_lens_dft_is_centred_unitary_dft():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16))
    ref = np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(x))) / 16
    assert rel_l2(O.lens_dft(x), ref) < 1e-14
    assert rel_l2(O.lens_dft(O.lens_dft(x), inverse=True), x) < 1e-14
    # a centred Gaussian maps to a centred real Gaussian
    g = O.source_gaussian(16, 1.0, 3.0)
    G = O.lens_dft(g)
    assert np.max(np.abs(G.imag)) < 1e-12 and np.argmax(np.abs(G)) == 8 * 16 + 8


def test_d2nn_identity_at_zero_phase_and_gradient():
    N, dx = 32, 0.03
    A = O.aperture(N, dx, 0.3048 * 2)
    assert A.sum() > 0 and A[0, 0] == 0 and A[N // 2, N // 2] == 1
    rng = np.random.default_rng(3)
    U = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    z = np.zeros((N, N))
    I, Z1, W2, V = O.d2nn_forward(A, z, z, U)
    assert np.max(np.abs(I - np.abs(A * U) ** 2)) < 1e-12
    # squared-error loss: central differences (eps = 1e-3 rad) against the adjoint, on 16 pixels per mask
    th1 = rng.normal(0, 0.1, (N, N))
    th2 = rng.normal(0, 0.1, (N, N))
    Iref = np.abs(O.source_gaussian(N, dx, 0.2)) ** 2 * A

    def loss(t1, t2):
        return O.intensity_loss(O.d2nn_forward(A, t1, t2, U)[0], Iref, 1, N * N)[0]

    I, Z1, W2, V = O.d2nn_forward(A, th1, th2, U)
    _, dLdI = O.intensity_loss(I, Iref, 1, N * N)
    g1, g2 = np.zeros((N, N)), np.zeros((N, N))
    gU = O.d2nn_backward(A, th1, th2, Z1, W2, V, dLdI, g1, g2)
    eps = 1e-3
    idx = rng.integers(0, N, size=(16, 2))
    scale = max(np.abs(g1).max(), np.abs(g2).max())
    for (j, i) in idx:
        for g, which in ((g1, 0), (g2, 1)):
            e = np.zeros((N, N))
            e[j, i] = eps
            if which == 0:
                fd = (loss(th1 + e, th2) - loss(th1 - e, th2)) / (2 * eps)
            else:
                fd = (loss(th1, th2 + e) - loss(th1, th2 - e)) / (2 * eps)
            assert abs(fd - g[j, i]) < 1e-5 * scale + 1e-6 * abs(fd)
    # gradient wrt the field
    e = np.zeros((N, N))
    j, i = N // 2, N // 2 + 1
    e[j, i] = 1e-6
    lf = lambda u: O.intensity_loss(O.d2nn_forward(A, th1, th2, u)[0], Iref, 1, N * N)[0]
    assert abs((lf(U + e) - lf(U - e)) / 2e-6 - gU[j, i].real) < 1e-6 * np.abs(gU).max()
    assert abs((lf(U + 1j * e) - lf(U - 1j * e)) / 2e-6 - gU[j, i].imag) < 1e-6 * np.abs(gU).max()
