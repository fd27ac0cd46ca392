"""The C-ABI library builds, loads and exports every symbol include/turbscreen.h declares; host-side
argument checks reject bad input before any CUDA call (CPU only, no kernel launches)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2604_07248_gb300 import binding as bd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "turbscreen.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ts_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_path_entry_points():
    names = declared_functions()
    for required in ("ts_plan_create", "ts_plan_destroy", "ts_make_screens", "ts_evolve_screens", "ts_propagate",
                     "ts_propagate_backward", "ts_moments_accumulate", "ts_moments_finalize", "ts_d2nn_forward",
                     "ts_d2nn_backward"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = bd.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
    # and the binding mirrors every declaration
    assert set(declared_functions()) <= set(bd.SIGNATURES)


def test_max_step_is_eq7_reading():
    # dz_max = (N dx / 2) sqrt(k^2 - kmax^2) / kmax, kmax = pi / dx  (approximately N dx^2 / lambda)
    for lam, N, dx in [(1.55e-6, 128, 2e-3), (1.55e-6, 1024, 5e-4), (1.064e-6, 1024, 3.4e-4)]:
        k = 2 * np.pi / lam
        kmax = np.pi / dx
        expect = 0.5 * N * dx * np.sqrt(k * k - kmax * kmax) / kmax
        assert abs(bd.max_step(lam, N, dx) - expect) < 1e-9 * expect
        assert abs(bd.max_step(lam, N, dx) / (N * dx * dx / lam) - 1) < 1e-3
    assert abs(bd.max_step(1.55e-6, 1024, 5e-4) - 165.1) < 0.2
    assert abs(bd.max_step(1.55e-6, 128, 2e-3) - 330.2) < 0.2


@pytest.mark.parametrize("kw,status", [
    (dict(N=100), 1),
    (dict(N=96), 1),
    (dict(dx=0.0), 1),
    (dict(lam=-1.0), 1),
    (dict(dz=[-5.0], cn2=[1e-15]), 1),
    (dict(dz=[10.0], cn2=[-1e-15]), 1),
    (dict(sh_levels=2), 1),
    (dict(max_batch=0), 1),
    (dict(dz=[1000.0], cn2=[1e-15]), 2),  # above the Eq. 7 limit of 330 m at N = 128, dx = 2 mm
    (dict(flags=bd.TS_PLAN_SPLIT_BF16), 6),  # the tensor-core passes exist for N = 1024 only
    (dict(alpha=3.0), 1),  # power law outside (3, 5)
    (dict(alpha=5.2), 1),
    (dict(alpha=4.3, A=-1.0), 1),
])
def test_plan_rejects_bad_arguments_before_touching_the_gpu(kw, status):
    args = dict(lam=1.55e-6, N=128, dx=2e-3, dz=[200.0], cn2=[1e-15], sh_levels=0, max_batch=1, flags=0,
                alpha=None, A=None)
    args.update(kw)
    with pytest.raises(bd.TsError) as ei:
        bd.Plan(args["lam"], args["N"], args["dx"], args["dz"], args["cn2"], sh_levels=args["sh_levels"],
                max_batch=args["max_batch"], flags=args["flags"], alpha=args["alpha"], A=args["A"])
    assert ei.value.status == status


def test_power_law_constant_host_function():
    # the library's A(alpha) (host code) against the oracle's, which the oracle tests pin to the
    # defining structure-function integral; NaN outside (3, 5)
    import oracle as O
    for a in (3.1, 3.5, 11 / 3, 4.0, 4.3, 4.41, 4.9):
        assert abs(bd.power_law_constant(a) / O.power_law_constant(a) - 1) < 1e-14
    assert np.isnan(bd.power_law_constant(3.0)) and np.isnan(bd.power_law_constant(5.0))


def test_status_strings_and_null_handling():
    lib = bd.load()
    for s in range(7):
        assert lib.ts_status_string(s)
    assert lib.ts_plan_destroy(None) == 0
    assert lib.ts_plan_device_bytes(None) == 0
    assert lib.ts_plan_device_status(None) == 1
    assert lib.ts_make_screens(None, 0, 0, 1, None, None, None) == 1
    assert lib.ts_propagate(None, None, 1, None, None, 1, 0, 0, 0, None, None, None) == 1
    assert b"need" in lib.ts_last_error()


def test_buffers_are_checked_before_their_pointers_cross_the_abi():
    # the C ABI takes raw pointers and sizes: the binding refuses a buffer of the wrong dtype, on the
    # wrong device or too small for the call, on the host, before anything is launched
    torch = pytest.importorskip("torch")
    bd._need(None, "optional", "float32", 10)  # optional buffers pass
    with pytest.raises(TypeError):
        bd._need(np.zeros(10, np.float32), "x", "float32", 10)
    with pytest.raises(TypeError):
        bd._need(torch.zeros(10, dtype=torch.float64), "x", "float32", 10)
    with pytest.raises(ValueError, match="CUDA"):
        bd._need(torch.zeros(10, dtype=torch.float32), "x", "float32", 10)
    with pytest.raises(TypeError):
        bd._need(torch.zeros(8, dtype=torch.int64), "ctr", ("int32", "uint32"), 8)
    if torch.cuda.is_available():  # pragma: no cover - the size check itself, on a CUDA tensor
        with pytest.raises(ValueError, match="needs 11"):
            bd._need(torch.zeros(10, dtype=torch.float32, device="cuda"), "x", "float32", 11)


def test_buffer_on_another_gpu_is_refused_before_its_pointer_crosses():
    # a tensor on cuda:1 handed to a call that runs on cuda:0 (a plan's device, or the device of the
    # call's other buffers) raises on the host; checked with stand-in tensors, so no GPU is needed
    torch = pytest.importorskip("torch")
    from unittest import mock

    def fake(dev, dtype=torch.complex64, n=64):
        t = mock.MagicMock(spec=torch.Tensor)
        t.dtype, t.is_cuda, t.device = dtype, True, torch.device("cuda", dev)
        t.numel.return_value = n
        return t

    bd._need(fake(0), "field", "complex64", 64, 0)  # same device passes
    bd._need(fake(1), "field", "complex64", 64)  # no device asked for: not checked
    with pytest.raises(ValueError, match="cuda:1.*cuda:0"):
        bd._need(fake(1), "field", "complex64", 64, 0)
    assert bd._device_of(fake(1), None, fake(1)) == 1
    with pytest.raises(ValueError, match="different GPUs"):
        bd._device_of(fake(0), fake(1))


def test_every_plan_entry_point_refuses_a_null_handle_without_a_gpu():
    # the boundary's error convention: a NULL plan or batch handle is TS_ERR_INVALID_ARG, returned
    # before any CUDA call (so this runs on a machine without a GPU); destroying NULL is a no-op
    lib = bd.load()
    N = None
    calls = {
        "ts_plan_device_status": (N,),
        "ts_plan_set_loss_scale": (N, 1.0),
        "ts_plan_tuning": (N,) + (None,) * 9,
        "ts_plan_tuning_candidates": (N, 0, None, None, None, None, None),
        "ts_plan_tuning_fused": (N, None, None, None),
        "ts_plan_tuning_columns": (N, None, None, None),
        "ts_plan_set_sources": (N, 1, None),
        "ts_make_sources": (N, None, 1, None),
        "ts_make_screens": (N, 1, 0, 1, None, None, None),
        "ts_evolve_screens": (N, 1, 0, 0, 0.9, 0.0, 0.0, 0.0, None, None, None, None, None),
        "ts_propagate": (N, None, 1, None, None, 1, 0, 0, 0, None, None, None),
        "ts_propagate_backward": (N, None, 1, None, None, 1, 0, 0, None),
        "ts_moments_accumulate": (N, None, 1, 1, 0, None, None, None, None, None),
        "ts_moments_finalize": (N, None, None, 1, 1, None, None, None, None, None, None),
        "ts_d2nn_forward": (N, None, 1, None, None, 0.3, None, 0, None, None, None, None),
        "ts_d2nn_backward": (N, 1, None, None, 0.3, None, 0, None, None, None, None, None, None),
        "ts_plan_timing": (N, 1, 4),
        "ts_plan_timing_read": (N, 0, None, None),
        "ts_batch_run": (N, None),
        "ts_batch_status": (N, None),
        "ts_batch_info": (N, None, None, None),
    }
    for name, args in calls.items():
        assert getattr(lib, name)(*args) == 1, name  # TS_ERR_INVALID_ARG
    assert lib.ts_plan_destroy(None) == bd.TS_OK and lib.ts_batch_destroy(None) == bd.TS_OK
    assert lib.ts_plan_device_bytes(None) == 0
