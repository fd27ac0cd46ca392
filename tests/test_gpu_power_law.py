"""GPU parity for the power-law media of Table S1 (ts_plan_create_psd): screens with and without
subharmonics, AR evolution and propagation through them, against the FP64 oracle with the same
power law and constant (relative L2 <= 1e-5)."""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - the gpu marker keeps these off CPU runs
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2604_07248_gb300 as ts  # noqa: E402

LAM = 1.55e-6
DEV = torch.device("cuda:0")
TOL = 1e-5


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.complex128 if np.iscomplexobj(a) else np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# (alpha, A): a general atmosphere, biological tissue with its A(alpha), an oceanic law with a caller's A
MEDIA = [(3.2, None), (4.3, None), (4.6, 0.05)]


@pytest.mark.parametrize("alpha,A", MEDIA)
@pytest.mark.parametrize("sh", [0, 3])
def test_power_law_screens_match_oracle(alpha, A, sh):
    N, dx, S = 256, 1e-3, 3
    dz, cn2 = [100.0] * S, [1e-14] * S
    plan = ts.Plan(LAM, N, dx, dz, cn2, l0=5e-3, L0=2.0, sh_levels=sh, max_batch=2, alpha=alpha, A=A)
    phi = torch.zeros((2, S, N, N), dtype=torch.float32, device=DEV)
    seed = 0x2604072480 + 11
    plan.make_screens(phi, seed, real_base=3, n_real=2)
    torch.cuda.synchronize()
    Aval = A if A is not None else O.power_law_constant(alpha)
    md = O.medium(LAM, N, dx, l0=5e-3, L0=2.0, alpha=alpha, A=Aval)
    got = phi.cpu().numpy()
    for r in range(2):
        for s in range(S):
            ref = O.make_screen(md, cn2[s], dz[s], sh, seed, s, 3 + r)
            assert rel_l2(got[r, s], ref) < TOL, (r, s, rel_l2(got[r, s], ref))


def test_power_law_ar_evolution_matches_oracle():
    N, dx, S, a_ar, alpha = 256, 1e-3, 2, 0.98, 4.3
    dz, cn2 = [100.0] * S, [1e-14] * S
    A = O.power_law_constant(alpha)
    md = O.medium(LAM, N, dx, l0=5e-3, L0=2.0, alpha=alpha, A=A)
    plan = ts.Plan(LAM, N, dx, dz, cn2, l0=5e-3, L0=2.0, sh_levels=3, max_batch=1, alpha=alpha)
    spec = torch.zeros((S, N, N), dtype=torch.complex64, device=DEV)
    sh = torch.zeros((S, 27), dtype=torch.complex128, device=DEV)
    phi = torch.zeros((S, N, N), dtype=torch.float32, device=DEV)
    seed, real = 31, 2
    ref = [O.screen_spectrum(md, cn2[s], dz[s], 3, seed, s, real, 0) for s in range(S)]
    for t in range(3):
        plan.evolve_screens(spec, phi, seed, t, a_ar, real=real, sh_state=sh)
        torch.cuda.synchronize()
        for s in range(S):
            if t > 0:
                ref[s] = O.ar_step(md, cn2[s], dz[s], 3, seed, s, real, t, a_ar, ref[s][0], ref[s][1])
            assert rel_l2(spec[s].cpu().numpy(), ref[s][0]) < TOL
            assert rel_l2(phi[s].cpu().numpy(), O.screen_from_spectrum(md, ref[s][0], ref[s][1])) < TOL


@pytest.mark.parametrize("N,dx,fused", [(512, 1e-3, False), (1024, 5e-4, True)])
def test_propagation_through_power_law_screens(N, dx, fused, monkeypatch):
    # biological-tissue law (alpha = 4.3) over 3 steps, screens regenerated from the seed; at N = 1024
    # through the fused persistent launch
    if N == 1024:
        monkeypatch.setenv("TS_FFT_E", "32")
        monkeypatch.setenv("TS_FUSED", "1" if fused else "0")
    alpha, S, dzv = 4.3, 3, 60.0
    plan = ts.Plan(LAM, N, dx, [dzv] * S, [2e-14] * S, l0=5e-3, L0=2.0, max_batch=1, alpha=alpha)
    plan.set_sources([0.01])
    U = torch.zeros((1, N, N), dtype=torch.complex64, device=DEV)
    plan.propagate(U, 1, flags=ts.TS_PROP_SOURCE, seed=44)
    plan.device_status()
    md = O.medium(LAM, N, dx, l0=5e-3, L0=2.0, alpha=alpha, A=O.power_law_constant(alpha))
    phis = np.stack([O.make_screen(md, 2e-14, dzv, 0, 44, s, 0) for s in range(S)])
    ref = O.propagate(md, [dzv] * S, phis, O.source_gaussian(N, dx, 0.01))
    assert rel_l2(U[0].cpu().numpy(), ref) < TOL, rel_l2(U[0].cpu().numpy(), ref)
