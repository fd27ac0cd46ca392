"""ts_make_screen_noalloc: one screen with no device allocation, for callers that cannot call
cudaMalloc where they need a screen (see include/turbscreen.h).

Collected last on purpose: it checks the entry point through the C ABI against ts_make_screens on two
calls in a row, and it must also pass when run alone in a fresh process."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2604_07248_gb300 import binding as bd  # noqa: E402

LAM = 1.55e-6
DEV = torch.device("cuda:0")
TOL = 1e-5


def rel_l2(a, b):
    return float(np.linalg.norm(a.astype(np.float64) - b) / np.linalg.norm(b))


def test_noalloc_screen_matches_plan_screens_on_two_calls():
    lib = bd.load()
    N, dx, S = 512, 1e-3, 4
    dz = [100.0, 80.0, 120.0, 60.0]
    cn2 = [1e-14, 3e-15, 2e-14, 5e-15]
    plan = bd.Plan(LAM, N, dx, dz, cn2, l0=5e-3, L0=10.0, max_batch=3)
    ref = torch.zeros((3, S, N, N), dtype=torch.float32, device=DEV)
    seed = 0x2604072480 + 7
    plan.make_screens(ref, seed, real_base=0, n_real=3)
    med = bd.Medium(LAM, 1.0, 5e-3, 10.0)
    grid = bd.Grid(N, dx)
    stream = torch.cuda.current_stream().cuda_stream
    out = torch.zeros((N, N), dtype=torch.float32, device=DEV)
    for screen, real in [(2, 1), (0, 2)]:  # two calls in a row reuse the same static scratch
        out.fill_(float("nan"))
        st = lib.ts_make_screen_noalloc(C.byref(med), C.byref(grid), dz[screen], cn2[screen], seed, screen, real,
                                        out.data_ptr(), stream)
        assert st == 0, lib.ts_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        want = ref[real, screen].cpu().numpy().astype(np.float64)
        assert np.isfinite(got).all()
        assert rel_l2(got, want) < TOL
        if screen == 2:  # and directly against the FP64 oracle for the first call
            import oracle as O
            md = O.medium(LAM, N, dx, l0=5e-3, L0=10.0)
            assert rel_l2(got, O.make_screen(md, cn2[screen], dz[screen], 0, seed, screen, real)) < TOL


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = bd.load()
    out = torch.zeros((4,), dtype=torch.float32, device=DEV)
    med = bd.Medium(LAM, 1.0, 5e-3, 10.0)
    st = lib.ts_make_screen_noalloc(C.byref(med), C.byref(bd.Grid(2048, 1e-3)), 100.0, 1e-15, 1, 0, 0,
                                    out.data_ptr(), None)
    assert st == 3 and b"exceeds" in lib.ts_last_error()
    st = lib.ts_make_screen_noalloc(C.byref(med), C.byref(bd.Grid(300, 1e-3)), 100.0, 1e-15, 1, 0, 0,
                                    out.data_ptr(), None)
    assert st == 1 and b"128, 256, 512, 1024, 2048" in lib.ts_last_error()
    st = lib.ts_make_screen_noalloc(C.byref(med), C.byref(bd.Grid(256, 1e-3)), 100.0, 1e-15, 1, 64, 0,
                                    out.data_ptr(), None)
    assert st == 1
