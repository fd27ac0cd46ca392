"""ctypes binding of libturbscreen.so (include/turbscreen.h).

Argument marshalling only: every function below forwards device pointers, sizes and the CUDA
stream handle to the C ABI, which runs every step of the path in the library's CUDA kernels.
There is no CPU path: if the library cannot be built or loaded, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading

from . import _build

_lock = threading.Lock()
_lib = None

TS_OK = 0
STATUS = {0: "ok", 1: "invalid argument", 2: "aliasing (Eq. 7)", 3: "workspace", 4: "CUDA error",
          5: "device timeout", 6: "unsupported"}

TS_PLAN_ALLOW_ALIASING = 1
TS_PLAN_SPLIT_BF16 = 2
TS_PLAN_TEST_STALL = 4
TS_PROP_SOURCE = 1
TS_PROP_INTENSITY = 2
TS_PROP_NO_FIELD = 4


class TsError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {detail}")
        self.status = status


class BatchInstance(C.Structure):
    _fields_ = [("plan", C.c_void_p), ("field", C.c_void_p), ("phasor", C.c_void_p), ("seed", C.c_uint64),
                ("real", C.c_uint32), ("source", C.c_int)]


TS_BATCH_TEST_STALL = 1
TS_BATCH_NO_TUNE = 2


class Medium(C.Structure):
    _fields_ = [("lambda_", C.c_double), ("n0", C.c_double), ("l0", C.c_double), ("L0", C.c_double)]


class Grid(C.Structure):
    _fields_ = [("N", C.c_int), ("dx", C.c_double)]


class Path(C.Structure):
    _fields_ = [("n_screens", C.c_int), ("dz", C.POINTER(C.c_double)), ("cn2", C.POINTER(C.c_double))]


# name -> (restype, argtypes); mirrors include/turbscreen.h
_P, _I, _D, _U32, _U64, _I64 = C.c_void_p, C.c_int, C.c_double, C.c_uint32, C.c_uint64, C.c_int64
SIGNATURES = {
    "ts_plan_create": (_I, [C.POINTER(_P), C.POINTER(Medium), C.POINTER(Grid), C.POINTER(Path), _I, _I, _I]),
    "ts_plan_create_psd": (_I, [C.POINTER(_P), C.POINTER(Medium), C.POINTER(Grid), C.POINTER(Path), _I, _I, _I, _D,
                                _D]),
    "ts_power_law_constant": (_D, [_D]),
    "ts_plan_destroy": (_I, [_P]),
    "ts_plan_device_status": (_I, [_P]),
    "ts_plan_set_loss_scale": (_I, [_P, _D]),
    "ts_plan_device_bytes": (C.c_size_t, [_P]),
    "ts_plan_tuning": (_I, [_P, C.POINTER(C.c_int), C.POINTER(C.c_float), C.POINTER(C.c_float),
                            C.POINTER(C.c_int), C.POINTER(C.c_float), C.POINTER(C.c_int), C.POINTER(C.c_float),
                            C.POINTER(C.c_int), C.POINTER(C.c_float)]),
    "ts_plan_tuning_candidates": (_I, [_P, _I, C.POINTER(C.c_int), _P, _P, _P, _P]),
    "ts_plan_tuning_fused": (_I, [_P, C.POINTER(C.c_int), C.POINTER(C.c_float), C.POINTER(C.c_float)]),
    "ts_plan_tuning_columns": (_I, [_P, C.POINTER(C.c_int), C.POINTER(C.c_float), C.POINTER(C.c_float)]),
    "ts_max_step": (_D, [C.POINTER(Medium), C.POINTER(Grid)]),
    "ts_cn2_hufnagel_valley": (_I, [_P, _I, _D, _D, _P]),
    "ts_adam_step": (_I, [_P, _P, _P, _P, C.c_longlong, _D, _D, _D, _D, _I, _P]),
    "ts_rytov_interval": (_I, [_P, _P, _I, _D, _D, _D, _P]),
    "ts_place_screens": (_I, [_P, _P, _I, C.POINTER(Medium), C.POINTER(Grid), _D, _P, _I, _D, _I, _P, _P, _P, _P]),
    "ts_plan_set_sources": (_I, [_P, _I, _P]),
    "ts_make_sources": (_I, [_P, _P, _I, _P]),
    "ts_make_screens": (_I, [_P, _U64, _U32, _I, _P, _P, _P]),
    "ts_evolve_screens": (_I, [_P, _U64, _U32, _U32, _D, _D, _D, _D, _P, _P, _P, _P, _P]),
    "ts_propagate": (_I, [_P, _P, _I, _P, _P, _I, _I, _U64, _U32, _P, _P, _P]),
    "ts_propagate_backward": (_I, [_P, _P, _I, _P, _P, _I, _U64, _U32, _P]),
    "ts_moments_accumulate": (_I, [_P, _P, _I, _I, _I64, _P, _P, _P, _P, _P]),
    "ts_moments_finalize": (_I, [_P, _P, _P, _I, _I64, _P, _P, _P, _P, _P, _P]),
    "ts_d2nn_forward": (_I, [_P, _P, _I, _P, _P, _D, _P, _I, _P, _P, _P, _P]),
    "ts_d2nn_backward": (_I, [_P, _I, _P, _P, _D, _P, _I, _P, _P, _P, _P, _P, _P]),
    "ts_philox4x32_10": (_I, [_P, _U32, _U32, _I, _P, _P]),
    "ts_tc_dft32": (_I, [_P, _P, _I, _I, _I, _D, _P, _P]),
    "ts_plan_timing": (_I, [_P, _I, _I]),
    "ts_plan_timing_read": (_I, [_P, _I, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "ts_make_screen_noalloc": (_I, [C.POINTER(Medium), C.POINTER(Grid), _D, _D, _U64, _U32, _U32, _P, _P]),
    "ts_batch_create": (_I, [C.POINTER(_P), C.POINTER(BatchInstance), _I, _D, _I]),
    "ts_batch_run": (_I, [_P, _P]),
    "ts_batch_status": (_I, [_P, _P]),
    "ts_batch_info": (_I, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_size_t)]),
    "ts_batch_tuning": (_I, [_P, C.POINTER(C.c_int), _P, _P, C.POINTER(C.c_int), C.POINTER(C.c_int),
                             C.POINTER(C.c_float), C.POINTER(C.c_float)]),
    "ts_batch_destroy": (_I, [_P]),
    "ts_status_string": (C.c_char_p, [_I]),
    "ts_last_error": (C.c_char_p, []),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libturbscreen.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"libturbscreen.so not found at {path}; run __graft_entry__.build()")
            lib = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(status: int, where: str):
    if status != TS_OK:
        detail = load().ts_last_error().decode()
        raise TsError(status, where, detail)


def _ptr(t) -> int | None:
    """Device pointer of a tensor (or None).  The C ABI reads raw memory, so lazily conjugated or
    non-contiguous views are rejected rather than passed with the wrong contents."""
    if t is None:
        return None
    if getattr(t, "is_conj", None) is not None and t.is_conj():
        raise ValueError("tensor has a pending conjugation (call .resolve_conj())")
    if getattr(t, "is_contiguous", None) is not None and not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _need(t, name: str, dtype, numel: int, device: int | None = None):
    """Checks a buffer before its raw pointer crosses the C ABI: a CUDA tensor of `dtype` (a torch
    dtype name, or a tuple of names any of which will do) holding at least `numel` elements, on GPU
    `device` when one is given.  The library receives only pointers and sizes, so an undersized or
    mistyped buffer, or one that lives on another GPU than the kernels run on, would be read or
    written out of bounds on the device; here it raises on the host instead.  None passes (optional
    buffers)."""
    if t is None:
        return
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    names = (dtype,) if isinstance(dtype, str) else tuple(dtype)
    if not any(t.dtype == getattr(torch, nm, None) for nm in names):
        raise TypeError(f"{name} must be torch.{' or torch.'.join(names)}, got {t.dtype}")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if device is not None and t.device.index != device:
        raise ValueError(f"{name} is on cuda:{t.device.index}, but the call runs on cuda:{device}")
    if t.numel() < numel:
        raise ValueError(f"{name} holds {t.numel()} elements, the call needs {numel}")


def _stream(stream, device: int | None = None) -> int | None:
    """The raw cudaStream_t of `stream`, or of `device`'s current stream when stream is None."""
    if stream is None:
        import torch
        return torch.cuda.current_stream(device).cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


def _on(device: int):
    """Context that makes `device` the current CUDA device for the duration of one library call (the
    library enqueues its work on the current device)."""
    import torch
    return torch.cuda.device(device)


def _device_of(*tensors) -> int:
    """The GPU index shared by the given tensors (None entries skipped); raises if they differ."""
    devs = {t.device.index for t in tensors if t is not None and getattr(t, "is_cuda", False)}
    if len(devs) > 1:
        raise ValueError(f"buffers of one call live on different GPUs: {sorted(devs)}")
    if not devs:
        import torch
        return torch.cuda.current_device()
    return devs.pop()


def max_step(lam, N, dx, n0=1.0) -> float:
    """Eq. 7 aliasing-limited step [m] for this wavelength and grid."""
    return load().ts_max_step(C.byref(Medium(lam, n0, 0.0, 0.0)), C.byref(Grid(N, dx)))


def adam_step(param, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """One Adam step on device float32 tensors (see ts_adam_step); t >= 1."""
    n = int(param.numel())
    dev = _device_of(param)
    for t_, nm in ((param, "param"), (grad, "grad"), (m, "m"), (v, "v")):
        _need(t_, nm, "float32", n, dev)
    with _on(dev):
        _check(load().ts_adam_step(_ptr(param), _ptr(grad), _ptr(m), _ptr(v), n, float(lr), float(beta1),
                                   float(beta2), float(eps), int(t), _stream(stream, dev)), "ts_adam_step")


def _host_f64(x):
    import numpy as np
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    return a, a.ctypes.data_as(C.c_void_p)


def cn2_hufnagel_valley(h, V=21.0, A=1.7e-14):
    """Hufnagel-Valley Cn^2 (S21) at heights h [m] (HV5/7: V = 21 m/s, A = 1.7e-14); numpy array."""
    import numpy as np
    ha, hp = _host_f64(np.atleast_1d(h))
    out = np.zeros_like(ha)
    _check(load().ts_cn2_hufnagel_valley(hp, int(ha.size), float(V), float(A), out.ctypes.data_as(C.c_void_p)),
           "ts_cn2_hufnagel_valley")
    return out


def rytov_interval(prof_z, prof_cn2, lam, z0, z1) -> float:
    """Rytov variance (S19) of [z0, z1] for a piecewise-linear sampled Cn^2 profile."""
    za, zp = _host_f64(prof_z)
    ca, cp = _host_f64(prof_cn2)
    out = C.c_double()
    _check(load().ts_rytov_interval(zp, cp, int(za.size), float(lam), float(z0), float(z1), C.byref(out)),
           "ts_rytov_interval")
    return out.value


def place_screens(prof_z, prof_cn2, lam, N, dx, L, rytov_limit, init_bounds=None, max_screens=64, n0=1.0):
    """Screen placement of Sec. 2.4 (see ts_place_screens): returns numpy arrays (dz, cn2, rytov)."""
    import numpy as np
    za, zp = _host_f64(prof_z)
    ca, cp = _host_f64(prof_cn2)
    ib = np.zeros(0) if init_bounds is None else np.asarray(init_bounds, dtype=np.float64)
    ia, ip = _host_f64(ib)
    dz, cn, ry = (np.zeros(int(max_screens)) for _ in range(3))
    n = C.c_int()
    _check(load().ts_place_screens(zp, cp, int(za.size), C.byref(Medium(lam, n0, 0.0, 0.0)), C.byref(Grid(N, dx)),
                                   float(L), ip if ia.size else None, int(ia.size), float(rytov_limit),
                                   int(max_screens), dz.ctypes.data_as(C.c_void_p), cn.ctypes.data_as(C.c_void_p),
                                   ry.ctypes.data_as(C.c_void_p), C.byref(n)), "ts_place_screens")
    k = n.value
    return dz[:k].copy(), cn[:k].copy(), ry[:k].copy()


def philox4x32_10(ctr, key0, key1, out, stream=None):
    """Philox4x32-10 words of n counters (ctr, out: device uint32 tensors of 4n words)."""
    n = ctr.numel() // 4
    dev = _device_of(ctr)
    _need(ctr, "ctr", ("int32", "uint32"), 4 * n, dev)  # 32-bit words
    _need(out, "out", ("int32", "uint32"), 4 * n, dev)
    with _on(dev):
        _check(load().ts_philox4x32_10(_ptr(ctr), int(key0), int(key1), n, _ptr(out), _stream(stream, dev)),
               "ts_philox4x32_10")


def make_screen_noalloc(phi, lam, N, dx, dz, cn2, seed, screen=0, real=0, n0=1.0, l0=0.0, L0=0.0, stream=None):
    """One screen (float32 [N, N] device tensor phi) without any device allocation; see
    ts_make_screen_noalloc in include/turbscreen.h."""
    L0v = float(L0) if (L0 is not None and math.isfinite(L0)) else 0.0
    med = Medium(float(lam), float(n0), float(l0), L0v)
    dev = _device_of(phi)
    _need(phi, "phi", "float32", int(N) * int(N), dev)
    with _on(dev):  # the scratch array's address is looked up on the current device
        _check(load().ts_make_screen_noalloc(C.byref(med), C.byref(Grid(int(N), float(dx))), float(dz), float(cn2),
                                             int(seed), int(screen), int(real), _ptr(phi), _stream(stream, dev)),
               "ts_make_screen_noalloc")


def tc_dft32(x, X, sign=-1, layout=0, err=None, timeout_s=1.0, stream=None):
    """Split-BF16 tensor-core 32-point DFTs of x [nvec, 32] complex64 into X (see ts_tc_dft32)."""
    import torch
    if err is None:
        err = torch.zeros(1, dtype=torch.int32, device=x.device)
    nvec = x.numel() // 32
    dev = _device_of(x)
    _need(x, "x", "complex64", 32 * nvec, dev)
    _need(X, "X", "complex64", 32 * nvec, dev)
    _need(err, "err", "int32", 1, dev)
    with _on(dev):
        _check(load().ts_tc_dft32(_ptr(x), _ptr(X), nvec, int(sign), int(layout), float(timeout_s), _ptr(err),
                                  _stream(stream, dev)),
               "ts_tc_dft32")
    return err


def power_law_constant(alpha: float) -> float:
    """A(alpha) of the power-law index PSD A Cn^2 kappa^-alpha (ts_power_law_constant; 0.0330 at 11/3)."""
    return load().ts_power_law_constant(float(alpha))


class Plan:
    """One medium + grid + path on the current CUDA device (ts_plan).  With `alpha` (and optionally
    `A`; default ts_power_law_constant(alpha)) the medium's index PSD is the power law of Table S1
    (ts_plan_create_psd), else the Kolmogorov modified von Karman PSD."""

    def __init__(self, lam, N, dx, dz, cn2, n0=1.0, l0=0.0, L0=0.0, sh_levels=0, max_batch=1, flags=0,
                 alpha=None, A=None):
        lib = load()
        dz = [float(x) for x in dz]
        cn2 = [float(x) for x in cn2]
        if len(dz) != len(cn2):
            raise ValueError("dz and cn2 need one entry per screen")
        self.N, self.dx, self.S, self.lam = int(N), float(dx), len(dz), float(lam)
        self.dz, self.cn2 = dz, cn2
        self.sh_levels, self.max_batch = int(sh_levels), int(max_batch)
        L0v = float(L0) if (L0 is not None and math.isfinite(L0)) else 0.0
        med = Medium(float(lam), float(n0), float(l0), L0v)
        grid = Grid(int(N), float(dx))
        dza = (C.c_double * len(dz))(*dz)
        cna = (C.c_double * len(cn2))(*cn2)
        path = Path(len(dz), dza, cna)
        h = C.c_void_p()
        if alpha is None and A is None:
            _check(lib.ts_plan_create(C.byref(h), C.byref(med), C.byref(grid), C.byref(path), int(sh_levels),
                                      int(max_batch), int(flags)), "ts_plan_create")
        else:
            a = 11.0 / 3.0 if alpha is None else float(alpha)
            A = float(A) if A is not None else lib.ts_power_law_constant(a)
            _check(lib.ts_plan_create_psd(C.byref(h), C.byref(med), C.byref(grid), C.byref(path), int(sh_levels),
                                          int(max_batch), int(flags), a, A), "ts_plan_create_psd")
        self._h = h
        import torch
        self.device = torch.cuda.current_device()  # the plan's tables and workspace live here

    @property
    def handle(self):
        return self._h

    def device_bytes(self) -> int:
        return load().ts_plan_device_bytes(self._h)

    def tuning(self):
        """(points per thread, us for E=16, us for E=32, concurrent field groups, us for 1/2/4 groups,
        column variant, us for E=32 with warp-owned columns, row variant, us for E=32 with shared
        phasor rows)."""
        e, a, b, g, v, w = C.c_int(), C.c_float(), C.c_float(), C.c_int(), C.c_int(), C.c_float()
        rv, rw = C.c_int(), C.c_float()
        us = (C.c_float * 3)()
        _check(load().ts_plan_tuning(self._h, C.byref(e), C.byref(a), C.byref(b), C.byref(g), us, C.byref(v),
                                     C.byref(w), C.byref(rv), C.byref(rw)), "ts_plan_tuning")
        return e.value, a.value, b.value, g.value, [us[0], us[1], us[2]], v.value, w.value, rv.value, rw.value

    def tuning_candidates(self):
        """The autotuner's candidate table: a list of (points per thread, column variant, row variant,
        us for one column + one row pass; 0 = not timed)."""
        n = C.c_int()
        _check(load().ts_plan_tuning_candidates(self._h, 0, C.byref(n), None, None, None, None),
               "ts_plan_tuning_candidates")
        e, cv, rv = (C.c_int * n.value)(), (C.c_int * n.value)(), (C.c_int * n.value)()
        us = (C.c_float * n.value)()
        _check(load().ts_plan_tuning_candidates(self._h, n.value, C.byref(n), e, cv, rv, us),
               "ts_plan_tuning_candidates")
        return [(e[i], cv[i], rv[i], us[i]) for i in range(n.value)]

    def tuning_columns(self):
        """(column variant in use, us per pass pair with column variant 2 (wide tiles), with variant 3
        (narrow tiles)), the last two timed under the chosen concurrent field groups (0 when not timed)."""
        v, a, b = C.c_int(), C.c_float(), C.c_float()
        _check(load().ts_plan_tuning_columns(self._h, C.byref(v), C.byref(a), C.byref(b)), "ts_plan_tuning_columns")
        return v.value, a.value, b.value

    def tuning_fused(self):
        """(fused, us per propagation with per-pass launches, us with the fused persistent launch)."""
        f, a, b = C.c_int(), C.c_float(), C.c_float()
        _check(load().ts_plan_tuning_fused(self._h, C.byref(f), C.byref(a), C.byref(b)), "ts_plan_tuning_fused")
        return bool(f.value), a.value, b.value

    def set_loss_scale(self, scale: float):
        """Factor on the D2NN receiver loss and its gradients (see ts_plan_set_loss_scale)."""
        _check(load().ts_plan_set_loss_scale(self._h, float(scale)), "ts_plan_set_loss_scale")

    def device_status(self):
        """Waits for the device and raises TsError (TS_ERR_DEVICE_TIMEOUT) if a bounded device wait of
        the plan's passes (tensor-core MMAs, or the TMA copies of the prefetching variants) ran out of its
        budget since the last call."""
        with _on(self.device):
            _check(load().ts_plan_device_status(self._h), "ts_plan_device_status")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            try:
                with _on(self.device):
                    load().ts_plan_destroy(self._h)
            except Exception:  # interpreter shutdown: torch may already be gone
                load().ts_plan_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def timing(self, enable: bool, capacity: int = 0):
        """Record CUDA events around each launch (kinds: 0 column pass, 1 row pass, 2 screens, 3 fused
        propagation)."""
        with _on(self.device):
            _check(load().ts_plan_timing(self._h, 1 if enable else 0, int(capacity)), "ts_plan_timing")

    def timing_read(self, kind: int):
        """(number of timed launches, summed device milliseconds) for one kernel kind."""
        n, ms = C.c_int(), C.c_double()
        _check(load().ts_plan_timing_read(self._h, int(kind), C.byref(n), C.byref(ms)), "ts_plan_timing_read")
        return n.value, ms.value

    def set_sources(self, w0):
        w = (C.c_double * len(w0))(*[float(x) for x in w0])
        with _on(self.device):
            _check(load().ts_plan_set_sources(self._h, len(w0), w), "ts_plan_set_sources")

    def _n2(self) -> int:
        return self.N * self.N

    def make_sources(self, field, B, stream=None):
        _need(field, "field", "complex64", int(B) * self._n2(), self.device)
        with _on(self.device):
            _check(load().ts_make_sources(self._h, _ptr(field), int(B), _stream(stream, self.device)), "ts_make_sources")

    def make_screens(self, phi, seed, real_base=0, n_real=1, phasor=None, stream=None):
        n = int(n_real) * self.S * self._n2()
        _need(phi, "phi", "float32", n, self.device)
        _need(phasor, "phasor", "complex64", n, self.device)
        with _on(self.device):
            _check(load().ts_make_screens(self._h, int(seed), int(real_base), int(n_real), _ptr(phi), _ptr(phasor),
                                          _stream(stream, self.device)), "ts_make_screens")

    def evolve_screens(self, spec, phi, seed, t, alpha, real=0, vx=0.0, vy=0.0, T=0.0, sh_state=None, phasor=None,
                       stream=None):
        n = self.S * self._n2()
        _need(spec, "spec", "complex64", n, self.device)
        _need(phi, "phi", "float32", n, self.device)
        _need(phasor, "phasor", "complex64", n, self.device)
        _need(sh_state, "sh_state", "complex128", self.S * 27, self.device)
        with _on(self.device):
            _check(load().ts_evolve_screens(self._h, int(seed), int(real), int(t), float(alpha), float(vx), float(vy),
                                            float(T), _ptr(spec), _ptr(sh_state), _ptr(phi), _ptr(phasor),
                                            _stream(stream, self.device)), "ts_evolve_screens")

    def propagate(self, field, B, phi=None, phi_group=1, flags=0, seed=0, real_base=0, intensity=None,
                  beam_sums=None, phasor=None, stream=None):
        self._need_path(field, "field", B, phi, phasor, phi_group)
        _need(intensity, "intensity", "float32", int(B) * self._n2(), self.device)
        _need(beam_sums, "beam_sums", "float64", 2 * int(B), self.device)
        with _on(self.device):
            _check(load().ts_propagate(self._h, _ptr(field), int(B), _ptr(phi), _ptr(phasor), int(phi_group), int(flags),
                                       int(seed), int(real_base), _ptr(intensity), _ptr(beam_sums), _stream(stream, self.device)),
                   "ts_propagate")

    def _need_path(self, field, name, B, phi, phasor, phi_group):
        """The field [B][N][N] and the screen sets [ceil(B / phi_group)][S][N][N] of a propagation."""
        B, g = int(B), max(1, int(phi_group))
        _need(field, name, "complex64", B * self._n2(), self.device)
        n = -(-B // g) * self.S * self._n2()
        _need(phi, "phi", "float32", n, self.device)
        _need(phasor, "phasor", "complex64", n, self.device)

    def propagate_backward(self, grad, B, phi=None, phi_group=1, seed=0, real_base=0, phasor=None, stream=None):
        self._need_path(grad, "grad", B, phi, phasor, phi_group)
        with _on(self.device):
            _check(load().ts_propagate_backward(self._h, _ptr(grad), int(B), _ptr(phi), _ptr(phasor), int(phi_group),
                                                int(seed), int(real_base), _stream(stream, self.device)), "ts_propagate_backward")

    def moments_accumulate(self, intensity, B, n_groups, count, mean, m2, beam_sums=None, beam_acc=None,
                           stream=None):
        """FP64 Welford merge of B intensities into the n_groups running (mean, m2); with beam_sums (the
        [B][2] sums of propagate) also the groups' running beam sums beam_acc [n_groups][2]."""
        _need(intensity, "intensity", "float32", int(B) * self._n2(), self.device)
        _need(mean, "mean", "float64", int(n_groups) * self._n2(), self.device)
        _need(m2, "m2", "float64", int(n_groups) * self._n2(), self.device)
        _need(beam_sums, "beam_sums", "float64", 2 * int(B), self.device)
        _need(beam_acc, "beam_acc", "float64", 2 * int(n_groups), self.device)
        with _on(self.device):
            _check(load().ts_moments_accumulate(self._h, _ptr(intensity), int(B), int(n_groups), int(count), _ptr(mean),
                                                _ptr(m2), _ptr(beam_sums), _ptr(beam_acc),
                                                _stream(stream, self.device)), "ts_moments_accumulate")

    def moments_finalize(self, mean, m2, n_groups, count, si_map=None, si_mean=None, si_center=None, beam_acc=None,
                         w_lt=None, stream=None):
        """SI map, plane-mean SI and on-axis SI per group; with beam_acc, the long-term radius w_lt [m]."""
        n = int(n_groups) * self._n2()
        _need(mean, "mean", "float64", n, self.device)
        _need(m2, "m2", "float64", n, self.device)
        _need(si_map, "si_map", "float64", n, self.device)
        _need(si_mean, "si_mean", "float64", int(n_groups), self.device)
        _need(si_center, "si_center", "float64", int(n_groups), self.device)
        _need(beam_acc, "beam_acc", "float64", 2 * int(n_groups), self.device)
        _need(w_lt, "w_lt", "float64", int(n_groups), self.device)
        with _on(self.device):
            _check(load().ts_moments_finalize(self._h, _ptr(mean), _ptr(m2), int(n_groups), int(count), _ptr(beam_acc),
                                              _ptr(si_map), _ptr(si_mean), _ptr(si_center), _ptr(w_lt),
                                              _stream(stream, self.device)), "ts_moments_finalize")

    def _need_d2nn(self, B, th1, th2, Iref, ws, intensity):
        n2, B = self._n2(), int(B)
        _need(th1, "th1", "float32", n2, self.device)
        _need(th2, "th2", "float32", n2, self.device)
        _need(Iref, "Iref", "float32", n2, self.device)
        _need(ws, "ws", "complex64", 3 * B * n2, self.device)
        _need(intensity, "intensity", "float32", B * n2, self.device)

    def d2nn_forward(self, U, B, th1, th2, aperture, Iref, kind, ws, intensity, loss, stream=None):
        _need(U, "U", "complex64", int(B) * self._n2(), self.device)
        self._need_d2nn(B, th1, th2, Iref, ws, intensity)
        _need(loss, "loss", "float64", 1, self.device)
        with _on(self.device):
            _check(load().ts_d2nn_forward(self._h, _ptr(U), int(B), _ptr(th1), _ptr(th2), float(aperture), _ptr(Iref),
                                          int(kind), _ptr(ws), _ptr(intensity), _ptr(loss), _stream(stream, self.device)),
                   "ts_d2nn_forward")

    def d2nn_backward(self, B, th1, th2, aperture, Iref, kind, ws, intensity, g_th1, g_th2, gU, stream=None):
        self._need_d2nn(B, th1, th2, Iref, ws, intensity)
        _need(g_th1, "g_th1", "float32", self._n2(), self.device)
        _need(g_th2, "g_th2", "float32", self._n2(), self.device)
        _need(gU, "gU", "complex64", int(B) * self._n2(), self.device)
        with _on(self.device):
            _check(load().ts_d2nn_backward(self._h, int(B), _ptr(th1), _ptr(th2), float(aperture), _ptr(Iref), int(kind),
                                           _ptr(ws), _ptr(intensity), _ptr(g_th1), _ptr(g_th2), _ptr(gU),
                                           _stream(stream, self.device)), "ts_d2nn_backward")


class Batch:
    """Uneven batch of instances propagated by one persistent launch (ts_batch_*)."""

    def __init__(self, instances, timeout_s=5.0, flags=0):
        """instances: list of dicts with keys plan, field, phasor (or None), seed, real, source."""
        arr = (BatchInstance * len(instances))()
        self.device = instances[0]["plan"].device if instances else None
        for i, d in enumerate(instances):
            pl = d["plan"]
            if pl.device != self.device:
                raise ValueError(f"instances[{i}].plan lives on cuda:{pl.device}, instance 0 on cuda:{self.device}")
            _need(d["field"], f"instances[{i}].field", "complex64", pl.N * pl.N, self.device)
            _need(d.get("phasor"), f"instances[{i}].phasor", "complex64", pl.S * pl.N * pl.N, self.device)
            arr[i].plan = pl.handle.value
            arr[i].field = _ptr(d["field"])
            arr[i].phasor = _ptr(d.get("phasor"))
            arr[i].seed = int(d.get("seed", 0))
            arr[i].real = int(d.get("real", 0))
            arr[i].source = 1 if d.get("source") else 0
        self._keep = [d["plan"] for d in instances]
        h = C.c_void_p()
        with _on(self.device):
            _check(load().ts_batch_create(C.byref(h), arr, len(instances), float(timeout_s), int(flags)),
                   "ts_batch_create")
        self._h = h

    def run(self, stream=None):
        with _on(self.device):
            _check(load().ts_batch_run(self._h, _stream(stream, self.device)), "ts_batch_run")

    def status(self, stream=None) -> int:
        """0, or the TS_ERR_* code the device reported (does not raise)."""
        with _on(self.device):
            return load().ts_batch_status(self._h, _stream(stream, self.device))

    def tuning(self):
        """The autotuner's choices: {N: points per thread}, item order, configurations timed, replay
        time of the default and of the chosen configuration (us)."""
        n, order, cand = C.c_int(), C.c_int(), C.c_int()
        sizes, ppt = (C.c_int * 5)(), (C.c_int * 5)()
        d, c = C.c_float(), C.c_float()
        _check(load().ts_batch_tuning(self._h, C.byref(n), sizes, ppt, C.byref(order), C.byref(cand), C.byref(d),
                                      C.byref(c)), "ts_batch_tuning")
        return {"points_per_thread": {int(sizes[i]): int(ppt[i]) for i in range(n.value)},
                "order": "largest grids first" if order.value == 1 else "caller's order",
                "candidates": cand.value, "us_default": round(d.value, 1), "us_chosen": round(c.value, 1)}

    def info(self):
        n, g, b = C.c_int(), C.c_int(), C.c_size_t()
        _check(load().ts_batch_info(self._h, C.byref(n), C.byref(g), C.byref(b)), "ts_batch_info")
        return {"items": n.value, "grid": g.value, "device_bytes": b.value}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().ts_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
