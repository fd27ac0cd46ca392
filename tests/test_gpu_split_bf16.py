"""Split-BF16 tensor-core variant of the propagation passes (TS_PLAN_SPLIT_BF16, N = 1024) against
the FP64 oracle and the FP32 passes.

Tolerance: relative L2 error <= 2e-3 per field, the accuracy the method allows for the split-BF16
DFT (hi.hi + hi.lo + lo.hi keeps about 16 bits per product).  Every check also asserts that the
tensor-core result differs from the FP32 passes, so the variant really ran."""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2604_07248_gb300 as ts  # noqa: E402

LAM = 1.55e-6
DEV = torch.device("cuda:0")
TOL = 2e-3


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.complex128 if np.iscomplexobj(a) else np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def cfield(B, N):
    return torch.zeros((B, N, N), dtype=torch.complex64, device=DEV)


def config3_plans(flags_list):
    N, dx, S = 1024, 5e-4, 16
    return [ts.Plan(LAM, N, dx, [62.5] * S, [1e-15] * S, l0=5e-3, L0=10.0, max_batch=8, flags=f) for f in flags_list]


def test_config3_split_bf16_matches_oracle_and_fp32():
    # N = 1024, dx = 0.5 mm, 16 screens of 62.5 m, Cn^2 = 1e-15, one AR step (alpha = 0.99), 8 beams
    # w0 = 1.0 + 0.25 b cm sharing the screens (B = 8, phi_group = 8, phasor screens)
    N, S, alpha = 1024, 16, 0.99
    seed = 0x2604072480 + 3
    tc, fp = config3_plans([ts.TS_PLAN_SPLIT_BF16, 0])
    w0 = [0.01 + 0.0025 * b for b in range(8)]
    spec = torch.zeros((S, N, N), dtype=torch.complex64, device=DEV)
    ph = torch.zeros((S, N, N), dtype=torch.complex64, device=DEV)
    fp.set_sources(w0)
    tc.set_sources(w0)
    fp.evolve_screens(spec, None, seed, 0, alpha, phasor=ph)
    fp.evolve_screens(spec, None, seed, 1, alpha, phasor=ph)
    U_tc, U_fp = cfield(8, N), cfield(8, N)
    tc.propagate(U_tc, 8, phasor=ph, phi_group=8, flags=ts.TS_PROP_SOURCE)
    fp.propagate(U_fp, 8, phasor=ph, phi_group=8, flags=ts.TS_PROP_SOURCE)
    tc.device_status()
    got, ref32 = U_tc.cpu().numpy(), U_fp.cpu().numpy()
    for b in range(8):
        r = rel_l2(got[b], ref32[b])
        assert 1e-8 < r < TOL, (b, r)
    md = O.medium(LAM, N, 5e-4, l0=5e-3, L0=10.0)
    phis = []
    for s in range(S):
        sp, _ = O.screen_spectrum(md, 1e-15, 62.5, 0, seed, s, 0, 0)
        sp, _ = O.ar_step(md, 1e-15, 62.5, 0, seed, s, 0, 1, alpha, sp)
        phis.append(O.screen_from_spectrum(md, sp))
    phis = np.stack(phis)
    for b in (0, 7):
        ref = O.propagate(md, [62.5] * S, phis, O.source_gaussian(N, 5e-4, w0[b]))
        assert rel_l2(got[b], ref) < TOL, (b, rel_l2(got[b], ref))


def test_split_bf16_vacuum_gaussian_matches_analytic_beam():
    # w0 = 1 cm over 1 km in 16 steps: W(L) = 5.03 cm, the analytic paraxial beam (piston-free)
    N, dx, S, w0, L = 1024, 5e-4, 16, 0.01, 1000.0
    plan = ts.Plan(LAM, N, dx, [L / S] * S, [0.0] * S, max_batch=1, flags=ts.TS_PLAN_SPLIT_BF16)
    plan.set_sources([w0])
    U = cfield(1, N)
    plan.propagate(U, 1, flags=ts.TS_PROP_SOURCE)
    plan.device_status()
    zR = np.pi * w0 ** 2 / LAM
    W = w0 * np.sqrt(1 + (L / zR) ** 2)
    R = L * (1 + (zR / L) ** 2)
    x = (np.arange(N) - N // 2) * dx
    r2 = x[None, :] ** 2 + x[:, None] ** 2
    ana = (w0 / W) * np.exp(-r2 / W ** 2 + 1j * 2 * np.pi / LAM * r2 / (2 * R) - 1j * np.arctan(L / zR))
    got = U[0].cpu().numpy()
    assert rel_l2(got, ana) < TOL, rel_l2(got, ana)
    # unitary steps: the energy of the source is kept
    e_in = np.sum(np.exp(-2 * r2 / w0 ** 2))
    assert abs(np.sum(np.abs(got.astype(np.complex128)) ** 2) / e_in - 1) < 1e-4


@pytest.mark.parametrize("groups", ["1", "2"])
def test_split_bf16_column_tiles_of_4_and_8_columns(groups, monkeypatch):
    # the column pass in tiles of 4 columns (one 128-vector group) or 8 (two groups): same result
    # against the FP32 passes within the split-BF16 tolerance, both transfer directions
    monkeypatch.setenv("TS_TC_COL_GROUPS", groups)
    N, S, B = 1024, 3, 2
    tc = ts.Plan(LAM, N, 5e-4, [62.5] * S, [1e-14] * S, l0=5e-3, L0=10.0, max_batch=B, flags=ts.TS_PLAN_SPLIT_BF16)
    fp = ts.Plan(LAM, N, 5e-4, [62.5] * S, [1e-14] * S, l0=5e-3, L0=10.0, max_batch=B)
    rng = np.random.default_rng(30)
    U0 = (rng.standard_normal((B, N, N)) + 1j * rng.standard_normal((B, N, N))).astype(np.complex64)
    out = []
    for p in (tc, fp):
        U = torch.from_numpy(U0).to(DEV)
        p.propagate(U, B, seed=8)
        g = torch.from_numpy(U0).to(DEV)
        p.propagate_backward(g, B, seed=8)
        torch.cuda.synchronize()
        out.append((U.cpu().numpy(), g.cpu().numpy()))
    tc.device_status()
    for b in range(B):
        for k in range(2):
            r = rel_l2(out[0][k][b], out[1][k][b])
            assert 1e-8 < r < TOL, (b, k, r)


def test_split_bf16_exact_transfer_given_screens_and_adjoint():
    # dx = 0.1 mm, dz = 2 m: the kappa^6 term exceeds 1e-7 rad, so the exact transfer function runs;
    # float screens given, then the adjoint with screens regenerated from the seed
    N, dx, S, B = 1024, 1e-4, 3, 2
    md = O.medium(LAM, N, dx, l0=2e-4, L0=1.0)
    plan = ts.Plan(LAM, N, dx, [2.0] * S, [1e-12] * S, l0=2e-4, L0=1.0, max_batch=B, flags=ts.TS_PLAN_SPLIT_BF16)
    seed = 21
    phis = np.stack([O.make_screen(md, 1e-12, 2.0, 0, seed, s, 0) for s in range(S)])
    rng = np.random.default_rng(12)
    U0 = (rng.standard_normal((B, N, N)) + 1j * rng.standard_normal((B, N, N))).astype(np.complex64)
    U = torch.from_numpy(U0).to(DEV)
    plan.propagate(U, B, phi=torch.from_numpy(phis.astype(np.float32))[None].to(DEV), phi_group=B)
    plan.device_status()
    got = U.cpu().numpy()
    for b in range(B):
        ref = O.propagate(md, [2.0] * S, phis.astype(np.float32).astype(np.float64), U0[b])
        assert rel_l2(got[b], ref) < TOL, (b, rel_l2(got[b], ref))
    g0 = (rng.standard_normal((B, N, N)) + 1j * rng.standard_normal((B, N, N))).astype(np.complex64)
    g = torch.from_numpy(g0).to(DEV)
    plan.propagate_backward(g, B, phi=None, seed=seed, real_base=0)
    x = torch.from_numpy(U0).to(DEV)
    plan.propagate(x, B, phi=None, seed=seed, real_base=0)
    plan.device_status()
    G, X = g.cpu().numpy(), x.cpu().numpy()
    for b in range(B):
        phib = np.stack([O.make_screen(md, 1e-12, 2.0, 0, seed, s, b) for s in range(S)])
        ref = O.propagate_adjoint(md, [2.0] * S, phib, g0[b])
        assert rel_l2(G[b], ref) < TOL, (b, rel_l2(G[b], ref))
        lhs = np.vdot(g0[b].astype(np.complex128), X[b].astype(np.complex128))
        rhs = np.vdot(G[b].astype(np.complex128), U0[b].astype(np.complex128))
        assert abs(lhs - rhs) < 1e-4 * np.linalg.norm(g0[b]) * np.linalg.norm(U0[b])


def test_split_bf16_intensity_and_beam_sums_match_fp32(monkeypatch):
    # moments path (intensity only, no field) and one- vs two-stream field groups
    N, S, B = 1024, 4, 4
    seed = 5
    plans = {}
    for streams in ("1", "2"):
        monkeypatch.setenv("TS_PROP_STREAMS", streams)
        plans[streams] = ts.Plan(LAM, N, 5e-4, [62.5] * S, [3e-15] * S, l0=5e-3, L0=10.0, max_batch=B,
                                 flags=ts.TS_PLAN_SPLIT_BF16)
    monkeypatch.setenv("TS_PROP_STREAMS", "1")
    fp = ts.Plan(LAM, N, 5e-4, [62.5] * S, [3e-15] * S, l0=5e-3, L0=10.0, max_batch=B)
    out = {}
    for name, p in (("tc1", plans["1"]), ("tc2", plans["2"]), ("fp", fp)):
        p.set_sources([0.01, 0.02])
        U = cfield(B, N)
        I = torch.zeros((B, N, N), dtype=torch.float32, device=DEV)
        sums = torch.zeros((B, 2), dtype=torch.float64, device=DEV)
        p.propagate(U, B, flags=ts.TS_PROP_SOURCE | ts.TS_PROP_INTENSITY | ts.TS_PROP_NO_FIELD, seed=seed,
                    real_base=3, intensity=I, beam_sums=sums)
        torch.cuda.synchronize()
        out[name] = (I.cpu().numpy(), sums.cpu().numpy())
    plans["1"].device_status()
    plans["2"].device_status()
    assert np.array_equal(out["tc1"][0], out["tc2"][0])  # same arithmetic per field on either stream layout
    for b in range(B):
        r = rel_l2(out["tc1"][0][b], out["fp"][0][b])
        assert 1e-9 < r < TOL, (b, r)
    assert np.allclose(out["tc1"][1], out["fp"][1], rtol=TOL, atol=0)
