"""FP64 CPU oracle for the split-step turbulence path (TurPy, arXiv 2604.07248).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()`` and by the
CPU-baseline leg of ``bench.py``.  The product package never imports it and it imports nothing
from the product package.  The numerics live in ``turb_oracle.c`` (plain C, double precision, its
own radix-2 FFT and its own Philox4x32-10); this module only compiles it with gcc and marshals
numpy arrays through ctypes.

Every function cites the passage of the paper it follows; the conventions chosen where the paper
is silent or garbled are listed at the top of ``turb_oracle.c``.  All functions are pinned by the
CPU tests (``tests/test_oracle_*.py``) except the inner-scale constant kappa_m = 2 pi / l0, a
convention of the paper itself (S17): parity unpinned for that constant alone.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "turb_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liborc.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile turb_oracle.c into oracle/_lib/liborc.so (gcc, -O2, no -ffast-math)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
             "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Medium(C.Structure):
    """Mirror of ``orc_medium``: wavelength, mean index, inner/outer scale, grid N and dx, and the
    power law alpha and constant A of the index PSD (0 = Kolmogorov 11/3 and 0.033)."""
    _fields_ = [("lambda_", C.c_double), ("n0", C.c_double), ("l0", C.c_double), ("L0", C.c_double),
                ("N", C.c_int), ("dx", C.c_double), ("alpha", C.c_double), ("A", C.c_double)]


def medium(lam, N, dx, n0=1.0, l0=0.0, L0=0.0, alpha=0.0, A=0.0) -> Medium:
    """A medium with the modified von Karman PSD (S17) or, with alpha (Table S1) and A given, the
    power law A Cn^2 (kappa^2 + kappa0^2)^(-alpha/2) exp(-kappa^2/kappa_m^2) (S12, S15)."""
    return Medium(float(lam), float(n0), float(l0), float(L0 if np.isfinite(L0) else 0.0), int(N), float(dx),
                  float(alpha), float(A))


def power_law_constant(alpha) -> float:
    """A(alpha) = Gamma(alpha - 1) cos(pi alpha / 2) / (4 pi^2): the constant for which the index PSD
    A Cn^2 kappa^-alpha has the structure function Cn^2 r^(alpha - 3) (3 < alpha < 5)."""
    return _load().orc_power_law_constant(float(alpha))


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            d, i, u32, u64, p = C.c_double, C.c_int, C.c_uint32, C.c_uint64, C.c_void_p
            pm = C.POINTER(Medium)
            sig = {
                "orc_philox4x32_10": (None, [p, p, p]),
                "orc_noise_grid": (None, [i, u64, u32, u32, u32, p]),
                "orc_noise_sh_all": (None, [u64, u32, u32, u32, p]),
                "orc_fft": (None, [i, p, i]),
                "orc_fft2": (None, [i, p, i]),
                "orc_phase_psd": (d, [pm, d, d, d]),
                "orc_power_law_constant": (d, [d]),
                "orc_psd_amplitude": (None, [pm, d, d, p]),
                "orc_sh_amplitude": (None, [pm, d, d, p]),
                "orc_sh_screen": (None, [pm, p, p]),
                "orc_screen_from_spectrum": (None, [pm, p, p, p]),
                "orc_screen_spectrum": (None, [pm, d, d, i, u64, u32, u32, u32, p, p]),
                "orc_make_screen": (None, [pm, d, d, i, u64, u32, u32, p]),
                "orc_ar_step": (None, [pm, d, d, i, u64, u32, u32, u32, d, d, d, d, p, p]),
                "orc_source_gaussian": (None, [i, d, d, p]),
                "orc_transfer": (None, [pm, d, p]),
                "orc_propagate": (None, [pm, i, p, p, p]),
                "orc_propagate_adjoint": (None, [pm, i, p, p, p]),
                "orc_welford_update": (None, [C.c_size_t, p, C.c_long, p, p]),
                "orc_welford_merge": (None, [C.c_size_t, C.c_long, p, p, C.c_long, p, p]),
                "orc_beam_sums": (None, [i, d, p, p, p]),
                "orc_lens_dft": (None, [i, p, i]),
                "orc_aperture": (None, [i, d, d, p]),
                "orc_d2nn_forward": (None, [i, p, p, p, p, p, p, p, p]),
                "orc_intensity_loss": (d, [C.c_size_t, p, p, i, d, p]),
                "orc_d2nn_backward": (None, [i, p, p, p, p, p, p, p, p, p, p]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------------------------
# random numbers
# ---------------------------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 (Salmon et al., SC'11) of one 4x32 counter under a 2x32 key."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    _load().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def noise_grid(N, seed, s, r, t=0) -> np.ndarray:
    """Complex Gaussian noise N_c(0,1) on the N x N spectral grid (Eq. 2, S16)."""
    out = np.zeros((N, N), np.complex128)
    _load().orc_noise_grid(N, seed, s, r, t, _ptr(out))
    return out


def noise_sh(seed, s, r, t=0) -> np.ndarray:
    """Subharmonic noise: 3 levels x 9 sub-grid cells (Eq. 2)."""
    out = np.zeros((3, 9), np.complex128)
    _load().orc_noise_sh_all(seed, s, r, t, _ptr(out))
    return out


# ---------------------------------------------------------------------------------------------
# DFT
# ---------------------------------------------------------------------------------------------
def fft(x, sign=-1) -> np.ndarray:
    """Unnormalised 1-D DFT by the oracle's own radix-2 FFT (sign -1 forward, +1 inverse sum)."""
    a = _c128(x).copy()
    _load().orc_fft(a.shape[-1], _ptr(a), sign)
    return a


def fft2(x, sign=-1) -> np.ndarray:
    a = _c128(x).copy()
    _load().orc_fft2(a.shape[-1], _ptr(a), sign)
    return a


# ---------------------------------------------------------------------------------------------
# screens
# ---------------------------------------------------------------------------------------------
def phase_psd(md: Medium, cn2, dz, kappa2) -> float:
    """Phi_phi(kappa) = 2 pi k^2 dz 0.033 Cn^2 (kappa^2+kappa0^2)^(-11/6) exp(-kappa^2/kappa_m^2) (S14, S17)."""
    return _load().orc_phase_psd(C.byref(md), cn2, dz, kappa2)


def psd_amplitude(md: Medium, cn2, dz) -> np.ndarray:
    """s(kappa) = sqrt(Phi_phi dkx dky) on the grid, s(0) = 0 (S16)."""
    out = np.zeros((md.N, md.N), np.float64)
    _load().orc_psd_amplitude(C.byref(md), cn2, dz, _ptr(out))
    return out


def sh_amplitude(md: Medium, cn2, dz) -> np.ndarray:
    out = np.zeros((3, 9), np.float64)
    _load().orc_sh_amplitude(C.byref(md), cn2, dz, _ptr(out))
    return out


def sh_screen(md: Medium, a) -> np.ndarray:
    """phi_SH from the 27 subharmonic coefficients (Eq. 2), term by term."""
    a = _c128(a)
    out = np.zeros((md.N, md.N), np.float64)
    _load().orc_sh_screen(C.byref(md), _ptr(a), _ptr(out))
    return out


def screen_spectrum(md: Medium, cn2, dz, sh_levels, seed, s, r, t=0):
    """Spectrum s*c and subharmonic coefficients of screen (s, r) drawn with AR step t."""
    spec = np.zeros((md.N, md.N), np.complex128)
    sh = np.zeros((3, 9), np.complex128)
    _load().orc_screen_spectrum(C.byref(md), cn2, dz, sh_levels, seed, s, r, t, _ptr(spec), _ptr(sh))
    return spec, (sh if sh_levels else None)


def screen_from_spectrum(md: Medium, spec, sh=None) -> np.ndarray:
    """phi = Re(IDFT_unnorm(spec)) + phi_SH - mean (S16, Eq. 3)."""
    spec = _c128(spec)
    out = np.zeros((md.N, md.N), np.float64)
    shp = None if sh is None else _c128(sh)
    _load().orc_screen_from_spectrum(C.byref(md), _ptr(spec), None if shp is None else _ptr(shp), _ptr(out))
    return out


def make_screen(md: Medium, cn2, dz, sh_levels, seed, s, r) -> np.ndarray:
    out = np.zeros((md.N, md.N), np.float64)
    _load().orc_make_screen(C.byref(md), cn2, dz, sh_levels, seed, s, r, _ptr(out))
    return out


def ar_step(md: Medium, cn2, dz, sh_levels, seed, s, r, t, alpha, spec, sh=None, vx=0.0, vy=0.0, T=0.0):
    """One AR(1) update of a screen spectrum (Eq. 4-5); returns new (spec, sh)."""
    spec = _c128(spec).copy()
    shc = None if sh is None else _c128(sh).copy()
    _load().orc_ar_step(C.byref(md), cn2, dz, sh_levels, seed, s, r, t, alpha, vx, vy, T, _ptr(spec),
                        None if shc is None else _ptr(shc))
    return spec, shc


# ---------------------------------------------------------------------------------------------
# propagation
# ---------------------------------------------------------------------------------------------
def source_gaussian(N, dx, w0) -> np.ndarray:
    """Collimated Gaussian U = exp(-r^2 / w0^2) centred on pixel (N/2, N/2) (S22)."""
    out = np.zeros((N, N), np.complex128)
    _load().orc_source_gaussian(N, dx, w0, _ptr(out))
    return out


def transfer(md: Medium, dz) -> np.ndarray:
    out = np.zeros((md.N, md.N), np.complex128)
    _load().orc_transfer(C.byref(md), dz, _ptr(out))
    return out


def propagate(md: Medium, dz, phi, U) -> np.ndarray:
    """Eq. 1 over S steps; phi is (S, N, N) or None (vacuum)."""
    dz = _f64(np.atleast_1d(dz))
    U = _c128(U).copy()
    ph = None if phi is None else _f64(phi)
    _load().orc_propagate(C.byref(md), len(dz), _ptr(dz), None if ph is None else _ptr(ph), _ptr(U))
    return U


def propagate_adjoint(md: Medium, dz, phi, g) -> np.ndarray:
    dz = _f64(np.atleast_1d(dz))
    g = _c128(g).copy()
    ph = None if phi is None else _f64(phi)
    _load().orc_propagate_adjoint(C.byref(md), len(dz), _ptr(dz), None if ph is None else _ptr(ph), _ptr(g))
    return g


# ---------------------------------------------------------------------------------------------
# moments
# ---------------------------------------------------------------------------------------------
class Welford:
    """Per-pixel running mean and M2 of intensity across realizations (S25, Welford)."""

    def __init__(self, shape):
        self.n = 0
        self.mean = np.zeros(shape, np.float64)
        self.M2 = np.zeros(shape, np.float64)

    def update(self, I):
        I = _f64(I)
        self.n += 1
        _load().orc_welford_update(I.size, _ptr(I), self.n, _ptr(self.mean), _ptr(self.M2))

    def merge(self, other: "Welford"):
        _load().orc_welford_merge(self.mean.size, self.n, _ptr(self.mean), _ptr(self.M2), other.n,
                                  _ptr(other.mean), _ptr(other.M2))
        self.n += other.n

    def si_map(self):
        """Scintillation index per pixel, population variance / mean^2 (S25)."""
        return (self.M2 / self.n) / (self.mean ** 2)


def beam_sums(N, dx, I):
    I = _f64(I)
    a, b = C.c_double(), C.c_double()
    _load().orc_beam_sums(N, dx, _ptr(I), C.byref(a), C.byref(b))
    return a.value, b.value


# ---------------------------------------------------------------------------------------------
# D2NN receiver
# ---------------------------------------------------------------------------------------------
def lens_dft(x, inverse=False) -> np.ndarray:
    a = _c128(x).copy()
    _load().orc_lens_dft(a.shape[-1], _ptr(a), 1 if inverse else 0)
    return a


def aperture(N, dx, diameter) -> np.ndarray:
    out = np.zeros((N, N), np.float64)
    _load().orc_aperture(N, dx, diameter, _ptr(out))
    return out


def d2nn_forward(A, th1, th2, U):
    """Receiver forward for one field; returns I, Z1, W2, V (Sec. 2.5, 4.1)."""
    N = U.shape[-1]
    A, th1, th2, U = _f64(A), _f64(th1), _f64(th2), _c128(U)
    I = np.zeros((N, N), np.float64)
    Z1, W2, V = (np.zeros((N, N), np.complex128) for _ in range(3))
    _load().orc_d2nn_forward(N, _ptr(A), _ptr(th1), _ptr(th2), _ptr(U), _ptr(I), _ptr(Z1), _ptr(W2), _ptr(V))
    return I, Z1, W2, V


def intensity_loss(I, Iref, kind, count):
    """MAE (kind 0, Sec. 2.5) or squared error (kind 1) summed and divided by count; also dL/dI."""
    I, Iref = _f64(I), _f64(Iref)
    g = np.zeros_like(I)
    L = _load().orc_intensity_loss(I.size, _ptr(I), _ptr(Iref), kind, float(count), _ptr(g))
    return L, g


def d2nn_backward(A, th1, th2, Z1, W2, V, dLdI, g_th1, g_th2):
    """Receiver adjoint; accumulates into g_th1/g_th2 in place and returns dL/dU."""
    N = V.shape[-1]
    A, th1, th2 = _f64(A), _f64(th1), _f64(th2)
    Z1, W2, V, dLdI = _c128(Z1), _c128(W2), _c128(V), _f64(dLdI)
    assert g_th1.dtype == np.float64 and g_th1.flags.c_contiguous
    assert g_th2.dtype == np.float64 and g_th2.flags.c_contiguous
    gU = np.zeros((N, N), np.complex128)
    _load().orc_d2nn_backward(N, _ptr(A), _ptr(th1), _ptr(th2), _ptr(Z1), _ptr(W2), _ptr(V), _ptr(dLdI),
                              _ptr(g_th1), _ptr(g_th2), _ptr(gU))
    return gU
