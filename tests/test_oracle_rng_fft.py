"""Pins for the oracle's random numbers and DFT (CPU only).

Philox4x32-10 against the generator's published known-answer vectors; Box-Muller noise against
the normal distribution; the radix-2 FFT against the brute-force DFT sum and numpy.fft.
"""
import os

import numpy as np
import pytest
from scipy import stats

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            w = [int(x, 16) for x in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat_rows())
def test_philox_known_answers(ctr, key, out):
    got = O.philox4x32_10(ctr, key)
    assert [int(x) for x in got] == out


def test_noise_is_standard_complex_gaussian():
    # Eq. 2 / S16: N_c(0,1); reading: real and imaginary parts each N(0,1), independent.
    c = np.concatenate([O.noise_grid(128, 0x2604072480, s, 3).ravel() for s in range(4)])
    re, im = c.real, c.imag
    n = re.size
    for part in (re, im):
        assert abs(part.mean()) < 5 / np.sqrt(n)
        assert abs(part.var() - 1.0) < 5 * np.sqrt(2.0 / n)
        assert stats.kstest(part, "norm").pvalue > 1e-4
    assert abs(np.corrcoef(re, im)[0, 1]) < 5 / np.sqrt(n)
    # the two samples that share one Philox call (bins m and m + N/2) are independent too
    g = O.noise_grid(128, 7, 0, 0)
    assert abs(np.corrcoef(g[:64].real.ravel(), g[64:].real.ravel())[0, 1]) < 5 / np.sqrt(64 * 128)


def test_noise_depends_on_every_counter_word():
    base = O.noise_grid(16, 11, 1, 2, 3)
    for args in [(12, 1, 2, 3), (11, 2, 2, 3), (11, 1, 3, 3), (11, 1, 2, 4)]:
        other = O.noise_grid(16, *args)
        assert np.mean(np.abs(other - base) > 0) > 0.99


def test_subharmonic_noise_distribution():
    c = np.concatenate([O.noise_sh(5, s, r).ravel() for s in range(40) for r in range(40)])
    for part in (c.real, c.imag):
        assert stats.kstest(part, "norm").pvalue > 1e-4
    # distinct from the grid noise of the same counters
    assert not np.allclose(O.noise_sh(5, 0, 0)[0, :2], O.noise_grid(16, 5, 0, 0)[0, :2])


@pytest.mark.parametrize("n", [2, 4, 8, 16, 32])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft_matches_bruteforce_dft(n, sign):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    k = np.arange(n)
    dft = np.exp(sign * 2j * np.pi * np.outer(k, k) / n) @ x
    assert np.max(np.abs(O.fft(x, sign) - dft)) <= 1e-13 * max(1.0, np.abs(dft).max())


@pytest.mark.parametrize("n", [64, 512, 2048])
def test_fft_matches_numpy(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = np.fft.fft(x)
    assert np.linalg.norm(O.fft(x, -1) - ref) / np.linalg.norm(ref) < 1e-14
    assert np.linalg.norm(O.fft(x, +1) - n * np.fft.ifft(x)) / np.linalg.norm(ref) < 1e-14


def test_fft2_matches_numpy_and_parseval():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((64, 64)) + 1j * rng.standard_normal((64, 64))
    X = O.fft2(x)
    assert np.linalg.norm(X - np.fft.fft2(x)) / np.linalg.norm(X) < 1e-14
    assert abs(np.sum(np.abs(X) ** 2) / 64 ** 2 - np.sum(np.abs(x) ** 2)) < 1e-11 * np.sum(np.abs(x) ** 2)
    back = O.fft2(X, +1) / 64 ** 2
    assert np.max(np.abs(back - x)) < 1e-13
