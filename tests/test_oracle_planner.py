"""Path-planning oracle (Sec. 2.4, S19-S21) against closed forms, and the library's host planner
against the oracle (CPU only: these are host functions)."""
import numpy as np
import pytest

from oracle import planner as P

LAM = 1.064e-6
K = 2 * np.pi / LAM


def test_s19_reduces_to_plane_wave_rytov_for_a_constant_profile():
    # int_0^L (1 - z/L)^(5/3) dz = 3 L / 8, so S19 = 3.27 * 3/8 k^(7/6) Cn2 L^(11/6) = 1.226 ... (S26's 1.23)
    for cn2, L in [(1e-15, 1000.0), (3e-14, 250.0), (5e-17, 20000.0)]:
        got = P.rytov_interval([0.0, 1.0], [cn2, cn2], LAM, 0.0, L)
        assert abs(got / (3.27 * 3 / 8 * K ** (7 / 6) * cn2 * L ** (11 / 6)) - 1) < 1e-9
        assert abs(got / (1.23 * cn2 * K ** (7 / 6) * L ** (11 / 6)) - 1) < 4e-3  # 1.23 is 1.22625 rounded


def test_s19_weights_the_start_of_the_interval():
    # a thin layer at the start of an interval counts (1 - z/dz)^(5/3) ~ 1, at the end ~ 0
    z = np.array([0.0, 10.0, 20.0, 980.0, 990.0, 1000.0])
    front = np.array([1e-14, 1e-14, 0.0, 0.0, 0.0, 0.0])
    back = front[::-1].copy()
    assert P.rytov_interval(z, front, LAM, 0, 1000) > 100 * P.rytov_interval(z, back, LAM, 0, 1000)


def test_hv57_gives_r0_5cm_and_theta0_7urad_at_half_a_micron():
    # the profile's name: r0 = 5 cm and isoplanatic angle 7 urad at 0.5 um, zenith (V = 21, A = 1.7e-14)
    h = np.linspace(0.0, 60e3, 600001)
    c = P.hv_cn2(h)
    dh = h[1] - h[0]
    k = 2 * np.pi / 0.5e-6
    mu0 = (c.sum() - 0.5 * (c[0] + c[-1])) * dh
    mu53 = ((c * h ** (5 / 3)).sum() - 0.5 * c[-1] * h[-1] ** (5 / 3)) * dh
    r0 = (0.423 * k * k * mu0) ** (-3 / 5)
    theta0 = (2.91 * k * k * mu53) ** (-3 / 5)
    assert 0.045 < r0 < 0.055, r0
    assert 6.5e-6 < theta0 < 7.5e-6, theta0
    assert P.hv_cn2(0.0) == pytest.approx(1.7e-14 + 2.7e-16, rel=1e-12)


def test_constant_profile_placement_has_the_closed_form_length():
    # each interval (before the Eq. 7 split) reaches the limit: 1.226 k^(7/6) Cn2 dz^(11/6) = limit
    cn2, L, lim = 2e-14, 3000.0, 0.05
    N, dx = 1024, 3e-3  # Eq. 7 limit 8.7 km: no Eq. 7 split
    dz, c, ry = P.place_screens([0.0, 1.0], [cn2, cn2], LAM, N, dx, L, lim)
    d_star = (lim / (3.27 * 3 / 8 * K ** (7 / 6) * cn2)) ** (6 / 11)
    assert len(dz) == int(np.ceil(L / d_star))
    assert np.allclose(dz[:-1], d_star, rtol=1e-8)
    assert abs(dz.sum() - L) < 1e-9 * L
    assert np.allclose(c, cn2, rtol=1e-9)
    assert np.all(ry <= lim * (1 + 1e-9))


@pytest.mark.parametrize("A,lim,L", [(1.7e-14, 0.02, 1500.0), (1e-13, 0.05, 5000.0), (5e-15, 0.01, 800.0)])
def test_placement_invariants_on_hv57(A, lim, L):
    z = np.linspace(0.0, L, 1001)
    c = P.hv_cn2(z, A=A)
    N, dx = 1024, 0.34e-3
    dz, cn, ry = P.place_screens(z, c, LAM, N, dx, L, lim, init_bounds=[L / 3, 2 * L / 3])
    assert abs(dz.sum() - L) < 1e-9 * L
    assert np.all(ry <= lim * (1 + 1e-6))
    assert np.all(dz <= P.max_step(LAM, N, dx) * (1 + 1e-12))
    # the strength each screen carries integrates back to the path's
    assert abs(np.sum(cn * dz) / P.path_integral(z, c, 0.0, L) - 1) < 1e-6


lib = pytest.importorskip("paper_2604_07248_gb300.binding")


def test_library_rytov_interval_matches_oracle():
    z = np.linspace(0.0, 3000.0, 301)
    c = P.hv_cn2(z, A=4e-14)
    rng = np.random.default_rng(3)
    for _ in range(20):
        z0, z1 = np.sort(rng.uniform(0.0, 3000.0, 2))
        ref = P.rytov_interval(z, c, LAM, z0, z1, n=200001)
        got = lib.rytov_interval(z, c, LAM, z0, z1)
        assert abs(got / ref - 1) < 1e-7, (z0, z1, got, ref)
    # the closed form on a constant profile
    got = lib.rytov_interval([0.0, 1.0], [1e-15, 1e-15], LAM, 0.0, 1000.0)
    assert abs(got / (3.27 * 3 / 8 * K ** (7 / 6) * 1e-15 * 1000.0 ** (11 / 6)) - 1) < 1e-12


def test_library_hv_profile_matches_oracle():
    h = np.linspace(0.0, 30e3, 3001)
    for V, A in [(21.0, 1.7e-14), (30.0, 1e-13), (0.0, 0.0)]:
        assert np.allclose(lib.cn2_hufnagel_valley(h, V, A), P.hv_cn2(h, V, A), rtol=1e-12, atol=0)


@pytest.mark.parametrize("A,lim,L,N,dx", [(1.7e-14, 0.02, 1500.0, 1024, 0.34e-3), (1e-13, 0.05, 5000.0, 512, 1e-3),
                                          (1e-15, 0.2, 1500.0, 1024, 0.34e-3), (3e-14, 0.005, 1000.0, 256, 2e-3)])
def test_library_placement_matches_oracle(A, lim, L, N, dx):
    z = np.linspace(0.0, L, 751)
    c = P.hv_cn2(z, A=A)
    dz, cn, ry = lib.place_screens(z, c, LAM, N, dx, L, lim, init_bounds=[0.25 * L], max_screens=256)
    dz_o, cn_o, ry_o = P.place_screens(z, c, LAM, N, dx, L, lim, init_bounds=[0.25 * L])
    assert len(dz) == len(dz_o)
    assert np.allclose(dz, dz_o, rtol=1e-6, atol=1e-9 * L)
    assert np.allclose(cn, cn_o, rtol=1e-6)
    assert np.allclose(ry, ry_o, rtol=1e-5)


def test_library_placement_errors():
    z = np.linspace(0.0, 1000.0, 11)
    c = P.hv_cn2(z)
    with pytest.raises(lib.TsError) as ei:
        lib.place_screens(z, c, LAM, 1024, 0.34e-3, 1000.0, 1e-6, max_screens=4)
    assert ei.value.status == 3
    with pytest.raises(lib.TsError):
        lib.place_screens(z[::-1], c, LAM, 1024, 0.34e-3, 1000.0, 0.1)
    with pytest.raises(lib.TsError):
        lib.place_screens(z, -c, LAM, 1024, 0.34e-3, 1000.0, 0.1)
