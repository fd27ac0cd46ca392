"""Edge and degenerate cases of the GPU path: a single screen, uneven screen sets, a plane wave in
vacuum, the pure-translation AR limit, unitarity of the propagator (P^H P = I), and empty inputs."""
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
TOL = 1e-5


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.complex128 if np.iscomplexobj(a) else np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_single_screen_path_forward_intensity_and_adjoint():
    # S = 1: first row pass, one column pass, last row pass (no middle pass)
    N, dx, dz, cn2, seed = 256, 1e-3, 120.0, 2e-14, 61
    md = O.medium(LAM, N, dx, l0=5e-3, L0=10.0)
    plan = ts.Plan(LAM, N, dx, [dz], [cn2], l0=5e-3, L0=10.0, max_batch=2)
    plan.set_sources([0.02, 0.0])  # Gaussian and plane wave
    U = torch.zeros((2, N, N), dtype=torch.complex64, device=DEV)
    I = torch.zeros((2, N, N), dtype=torch.float32, device=DEV)
    plan.propagate(U, 2, flags=ts.TS_PROP_SOURCE | ts.TS_PROP_INTENSITY, seed=seed, intensity=I)
    g = U.clone()
    plan.propagate_backward(g, 2, seed=seed)
    torch.cuda.synchronize()
    for b, w0 in enumerate((0.02, 0.0)):
        phis = O.make_screen(md, cn2, dz, 0, seed, 0, b)[None]
        src = O.source_gaussian(N, dx, w0) if w0 > 0 else np.ones((N, N), complex)
        ref = O.propagate(md, [dz], phis, src)
        assert rel_l2(U[b].cpu().numpy(), ref) < TOL
        assert rel_l2(I[b].cpu().numpy(), np.abs(ref) ** 2) < 2 * TOL
        # the adjoint of the forward result comes back to the source (P^H P = I)
        assert rel_l2(g[b].cpu().numpy(), src) < TOL


@pytest.mark.parametrize("B,phi_group", [(5, 2), (3, 8), (4, 4)])
def test_uneven_screen_sets_match_oracle(B, phi_group):
    # B not a multiple of phi_group (the last set is shared by fewer fields) and phi_group > B;
    # B = max_batch
    N, dx, S = 128, 2e-3, 3
    G = (B + phi_group - 1) // phi_group
    md = O.medium(LAM, N, dx, l0=5e-3, L0=10.0)
    plan = ts.Plan(LAM, N, dx, [150.0] * S, [1e-14] * S, l0=5e-3, L0=10.0, max_batch=B)
    phis = np.stack([np.stack([O.make_screen(md, 1e-14, 150.0, 0, 70, s, g) for s in range(S)]) for g in range(G)])
    rng = np.random.default_rng(71)
    U0 = (rng.standard_normal((B, N, N)) + 1j * rng.standard_normal((B, N, N))).astype(np.complex64)
    U = torch.from_numpy(U0).to(DEV)
    plan.propagate(U, B, phi=torch.from_numpy(phis.astype(np.float32)).to(DEV), phi_group=phi_group)
    torch.cuda.synchronize()
    got = U.cpu().numpy()
    for b in range(B):
        ref = O.propagate(md, [150.0] * S, phis[b // phi_group].astype(np.float32).astype(np.float64), U0[b])
        assert rel_l2(got[b], ref) < TOL, (b, rel_l2(got[b], ref))


def test_plane_wave_in_vacuum_stays_a_plane_wave():
    # U = 1 is the DC mode: H(0) = 1 / N^2 times the N^2 of the forward transform, no screen
    N, dx, S = 512, 1e-3, 6
    plan = ts.Plan(LAM, N, dx, [150.0] * S, [0.0] * S, max_batch=1)
    plan.set_sources([0.0])
    U = torch.zeros((1, N, N), dtype=torch.complex64, device=DEV)
    plan.propagate(U, 1, flags=ts.TS_PROP_SOURCE)
    torch.cuda.synchronize()
    u = U[0].cpu().numpy()
    assert np.max(np.abs(u - 1.0)) < 1e-5


@pytest.mark.parametrize("cn2", [0.0, 3e-14])
def test_propagator_is_unitary(cn2):
    # |H| = 1 on the grid (no evanescent bins) and |exp(i phi)| = 1: P^H P x = x for any x
    N, dx, S = 256, 1e-3, 4
    plan = ts.Plan(LAM, N, dx, [100.0] * S, [cn2] * S, l0=5e-3, L0=10.0, max_batch=3)
    rng = np.random.default_rng(72)
    X = (rng.standard_normal((3, N, N)) + 1j * rng.standard_normal((3, N, N))).astype(np.complex64)
    U = torch.from_numpy(X).to(DEV)
    plan.propagate(U, 3, seed=9, real_base=4)
    e_out = float(U.abs().pow(2).sum().item())
    plan.propagate_backward(U, 3, seed=9, real_base=4)
    torch.cuda.synchronize()
    assert abs(e_out / float(np.sum(np.abs(X.astype(np.complex128)) ** 2)) - 1) < 1e-5
    for b in range(3):
        assert rel_l2(U[b].cpu().numpy(), X[b]) < TOL


def test_ar_with_alpha_one_is_a_pure_translation():
    # alpha = 1 with an integer-pixel wind displacement (vx T = 2 dx, vy T = -3 dx) shifts the
    # screen exactly (Eq. 4): phi_1 = roll(phi_0); independent of the oracle
    N, dx, S = 256, 1e-3, 2
    plan = ts.Plan(LAM, N, dx, [100.0] * S, [1e-14] * S, l0=5e-3, L0=10.0, max_batch=1)
    spec = torch.zeros((S, N, N), dtype=torch.complex64, device=DEV)
    phi0 = torch.zeros((S, N, N), dtype=torch.float32, device=DEV)
    phi1 = torch.zeros_like(phi0)
    T = 1e-3
    vx, vy = 2 * dx / T, -3 * dx / T
    plan.evolve_screens(spec, phi0, 12, 0, 1.0, vx=vx, vy=vy, T=T)
    plan.evolve_screens(spec, phi1, 12, 1, 1.0, vx=vx, vy=vy, T=T)
    torch.cuda.synchronize()
    a, b = phi0.cpu().numpy(), phi1.cpu().numpy()
    for s in range(S):
        # a displacement (vx, vy) T moves the screen content to larger x by 2 pixels, smaller y by 3
        shifted = np.roll(a[s], (-3, 2), axis=(0, 1))
        assert rel_l2(b[s], shifted) < 1e-5, rel_l2(b[s], shifted)


def test_empty_and_oversized_requests_are_rejected():
    plan = ts.Plan(LAM, 128, 2e-3, [100.0], [1e-15], max_batch=2)
    U = torch.zeros((3, 128, 128), dtype=torch.complex64, device=DEV)  # room for B = 3: the library refuses it
    for B in (0, -1, 3):
        with pytest.raises(ts.TsError):
            plan.propagate(U, B)
    phi = torch.zeros((1, 1, 128, 128), dtype=torch.float32, device=DEV)
    with pytest.raises(ts.TsError):
        plan.make_screens(phi, 1, n_real=0)
    with pytest.raises(ts.TsError):
        plan.propagate(U, 1, phi_group=0)


def test_undersized_or_mistyped_buffers_are_refused_on_the_host():
    # the binding checks every buffer against the call's sizes before its pointer reaches the
    # library, so a short field, a missing screen set or a wrong dtype never reaches a kernel
    N, S = 256, 2
    plan = ts.Plan(LAM, N, 1e-3, [100.0] * S, [1e-14] * S, l0=5e-3, L0=10.0, max_batch=4)
    U = torch.zeros((3, N, N), dtype=torch.complex64, device=DEV)
    with pytest.raises(ValueError, match="field"):
        plan.propagate(U, 4, seed=1)  # 3 of the 4 fields
    one = torch.zeros((1, 1, N, N), dtype=torch.complex64, device=DEV)
    with pytest.raises(ValueError, match="phasor"):
        plan.propagate(U, 3, phasor=one, phi_group=3)  # 1 of the S = 2 screens of the set
    with pytest.raises(TypeError, match="field"):
        plan.propagate(U.to(torch.complex128), 3, seed=1)
    with pytest.raises(ValueError, match="spec"):
        plan.evolve_screens(torch.zeros((1, N, N), dtype=torch.complex64, device=DEV), None, 1, 0, 0.99,
                            phasor=torch.zeros((S, N, N), dtype=torch.complex64, device=DEV))
    with pytest.raises(ValueError, match="mean"):
        plan.moments_accumulate(torch.zeros((4, N, N), dtype=torch.float32, device=DEV), 4, 2, 0,
                                torch.zeros((1, N, N), dtype=torch.float64, device=DEV),
                                torch.zeros((2, N, N), dtype=torch.float64, device=DEV))
    with pytest.raises(ValueError, match="grad"):
        plan.propagate_backward(U, 4, seed=1)
    # nothing was launched: the plan works as before
    plan.propagate(U, 3, seed=1)
    torch.cuda.synchronize()
    plan.device_status()
    assert bool(torch.isfinite(torch.view_as_real(U)).all())
    plan.close()
