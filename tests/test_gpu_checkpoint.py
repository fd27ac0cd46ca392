"""Checkpoint and resume.  The state of a Monte Carlo run is (seed, next realization, the FP64
Welford accumulators) and that of an AR run (spectra, subharmonic coefficients, next time step):
the screens of any realization and step come from Philox counters, so nothing else is needed to
continue.  A run stopped after some calls, its state copied to the host, the plan destroyed and a
new one created from the same parameters, must end bit for bit where the uninterrupted run ends."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - the gpu marker keeps these off CPU runs
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2604_07248_gb300 as ts  # noqa: E402

LAM = 1.55e-6
DEV = torch.device("cuda:0")


def _mc_plan(N, dx, S, B):
    plan = ts.Plan(LAM, N, dx, [150.0] * S, [3e-14] * S, l0=5e-3, L0=10.0, sh_levels=3, max_batch=B)
    plan.set_sources([0.0, 0.03])  # plane wave and Gaussian sharing each realization's screens
    return plan


def _mc_calls(plan, calls, first, seed, B, N, mean, m2, count):
    """Calls first..first+calls-1 of the run: B / 2 realizations x 2 sources each."""
    U = torch.zeros((B, N, N), dtype=torch.complex64, device=DEV)
    I = torch.zeros((B, N, N), dtype=torch.float32, device=DEV)
    for c in range(first, first + calls):
        plan.propagate(U, B, phi_group=2, flags=ts.TS_PROP_SOURCE | ts.TS_PROP_INTENSITY, seed=seed,
                       real_base=c * (B // 2), intensity=I)
        plan.moments_accumulate(I, B, 2, count, mean, m2)
        count += B // 2
    return count


def _finalize(plan, mean, m2, count):
    si_map = torch.zeros_like(mean)
    si_mean = torch.zeros(2, dtype=torch.float64, device=DEV)
    si_c = torch.zeros(2, dtype=torch.float64, device=DEV)
    plan.moments_finalize(mean, m2, 2, count, si_map=si_map, si_mean=si_mean, si_center=si_c)
    torch.cuda.synchronize()
    plan.device_status()
    return si_map, si_mean, si_c


@pytest.mark.parametrize("N,dx", [(128, 2e-3), (1024, 5e-4)])
def test_monte_carlo_resumes_bit_for_bit(N, dx):
    S, B, calls, stop, seed = 3, 8, 4, 2, 0x2604072480 + 2
    plan = _mc_plan(N, dx, S, B)
    mean = torch.zeros((2, N, N), dtype=torch.float64, device=DEV)
    m2 = torch.zeros_like(mean)
    count = _mc_calls(plan, calls, 0, seed, B, N, mean, m2, 0)
    ref = (mean.clone(), m2.clone()) + _finalize(plan, mean, m2, count)
    plan.close()

    plan = _mc_plan(N, dx, S, B)
    mean = torch.zeros((2, N, N), dtype=torch.float64, device=DEV)
    m2 = torch.zeros_like(mean)
    count = _mc_calls(plan, stop, 0, seed, B, N, mean, m2, 0)
    torch.cuda.synchronize()
    state = (mean.cpu().numpy().copy(), m2.cpu().numpy().copy(), count, stop)  # the checkpoint
    plan.close()
    del mean, m2
    torch.cuda.synchronize()

    plan = _mc_plan(N, dx, S, B)
    mean = torch.from_numpy(state[0]).to(DEV)
    m2 = torch.from_numpy(state[1]).to(DEV)
    count = _mc_calls(plan, calls - state[3], state[3], seed, B, N, mean, m2, state[2])
    got = (mean, m2) + _finalize(plan, mean, m2, count)
    plan.close()
    for a, b in zip(got, ref):
        assert torch.equal(a, b)


def _ar_plan(N, dx, S):
    return ts.Plan(LAM, N, dx, [100.0] * S, [1e-14] * S, l0=5e-3, L0=10.0, sh_levels=3, max_batch=1)


def _ar_steps(plan, t0, t1, spec, sh, phi, ph, seed, real, alpha, wind):
    for t in range(t0, t1):
        plan.evolve_screens(spec, phi, seed, t, alpha, real=real, vx=wind[0], vy=wind[1], T=wind[2], sh_state=sh,
                            phasor=ph)


@pytest.mark.parametrize("N,dx", [(256, 1e-3), (1024, 5e-4)])
def test_ar_evolution_resumes_bit_for_bit(N, dx):
    # AR(1) with wind tilt and subharmonics; the screens of the last step and a beam propagated
    # through them must be identical after a restart from the host copy of the state
    S, T, stop, seed, real, alpha, wind = 3, 6, 3, 41, 2, 0.99, (2.0, -1.0, 1e-3)

    def fresh():
        return (torch.zeros((S, N, N), dtype=torch.complex64, device=DEV),
                torch.zeros((S, 27), dtype=torch.complex128, device=DEV),
                torch.zeros((S, N, N), dtype=torch.float32, device=DEV),
                torch.zeros((S, N, N), dtype=torch.complex64, device=DEV))

    def beam(plan, ph):
        plan.set_sources([0.02])
        U = torch.zeros((1, N, N), dtype=torch.complex64, device=DEV)
        plan.propagate(U, 1, phasor=ph, flags=ts.TS_PROP_SOURCE)
        return U

    plan = _ar_plan(N, dx, S)
    spec, sh, phi, ph = fresh()
    _ar_steps(plan, 0, T, spec, sh, phi, ph, seed, real, alpha, wind)
    ref = (spec, sh, phi, ph, beam(plan, ph))
    torch.cuda.synchronize()
    plan.close()

    plan = _ar_plan(N, dx, S)
    spec, sh, phi, ph = fresh()
    _ar_steps(plan, 0, stop, spec, sh, phi, ph, seed, real, alpha, wind)
    torch.cuda.synchronize()
    state = (spec.cpu().numpy().copy(), sh.cpu().numpy().copy(), stop)  # the checkpoint
    plan.close()
    del spec, sh
    torch.cuda.synchronize()

    plan = _ar_plan(N, dx, S)
    spec = torch.from_numpy(state[0]).to(DEV)
    sh = torch.from_numpy(state[1]).to(DEV)
    _, _, phi, ph = fresh()
    _ar_steps(plan, state[2], T, spec, sh, phi, ph, seed, real, alpha, wind)
    got = (spec, sh, phi, ph, beam(plan, ph))
    torch.cuda.synchronize()
    plan.device_status()
    plan.close()
    for a, b in zip(got, ref):
        assert torch.equal(a, b)
    assert np.isfinite(ref[2].cpu().numpy()).all()
