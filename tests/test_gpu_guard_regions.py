"""Guard regions around every buffer the kernels write.  Each output sits inside a larger allocation
whose margins (32 KiB on each side) hold a sentinel; after the call the margins must be untouched.
An out-of-bounds store near a buffer (a persistent grid's last stride, a TMA box or bulk copy past
the end, a ragged tail, a wrong field or row index at the edge of a batch) changes them.  The cases
use ragged batches (B = 3, not a multiple of any tile or group count) on every propagation variant."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - the gpu marker keeps these off CPU runs
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2604_07248_gb300 as ts  # noqa: E402

LAM = 1.55e-6
DEV = torch.device("cuda:0")
MARGIN_BYTES = 32768
SENTINEL = {torch.complex64: complex(12345.678, -9876.5), torch.complex128: complex(-2.5e7, 3.25e9),
            torch.float32: -31415.926, torch.float64: 2.718281828e11}


class Guarded:
    """A tensor of `shape` inside an allocation with sentinel margins (the view starts 32 KiB into
    the allocation, so it keeps every alignment the library asks for)."""

    def __init__(self, shape, dtype, init=None):
        esize = torch.empty((), dtype=dtype).element_size()
        self.pad = MARGIN_BYTES // esize
        self.n = int(np.prod(shape))
        self.dtype = dtype
        self.base = torch.full((self.n + 2 * self.pad,), SENTINEL[dtype], dtype=dtype, device=DEV)
        self.t = self.base[self.pad:self.pad + self.n].view(shape)
        if init is None:
            self.t.zero_()
        else:
            self.t.copy_(init)

    def margins_intact(self):
        s = torch.tensor(SENTINEL[self.dtype], dtype=self.dtype, device=DEV)
        head, tail = self.base[:self.pad], self.base[self.pad + self.n:]
        return bool(torch.all(head == s)) and bool(torch.all(tail == s))


def _env(monkeypatch, **kv):
    for k, v in kv.items():
        monkeypatch.setenv(k, str(v))


def _random_field(B, N, seed):
    rng = np.random.default_rng(seed)
    return torch.from_numpy((rng.standard_normal((B, N, N)) + 1j * rng.standard_normal((B, N, N))).astype(np.complex64))


def _propagation_cases(plan, N, S, B, phasor):
    """Forward from sources and from a field, to the intensity with beam sums, and the adjoint."""
    plan.set_sources([0.01 + 0.002 * b for b in range(B)])
    outs = []
    U = Guarded((B, N, N), torch.complex64)
    plan.propagate(U.t, B, phasor=phasor, phi_group=B, flags=ts.TS_PROP_SOURCE)
    outs.append(U)
    V = Guarded((B, N, N), torch.complex64, _random_field(B, N, 3))
    I = Guarded((B, N, N), torch.float32)
    sums = Guarded((B, 2), torch.float64)
    plan.propagate(V.t, B, phasor=phasor, phi_group=B, flags=ts.TS_PROP_INTENSITY, intensity=I.t, beam_sums=sums.t)
    outs += [V, I, sums]
    G = Guarded((B, N, N), torch.complex64, _random_field(B, N, 4))
    plan.propagate_backward(G.t, B, phasor=phasor, phi_group=B)
    outs.append(G)
    torch.cuda.synchronize()
    plan.device_status()
    return outs


def _phasors(plan, N, S, seed=7):
    phi = torch.zeros((1, S, N, N), dtype=torch.float32, device=DEV)
    ph = Guarded((1, S, N, N), torch.complex64)
    plan.make_screens(phi, seed, n_real=1, phasor=ph.t)
    return ph


@pytest.mark.parametrize("N,dx,colv,fused", [(1024, 5e-4, 2, 0), (1024, 5e-4, 3, 0), (1024, 5e-4, 2, 1),
                                             (512, 1e-3, 2, 0), (512, 1e-3, 3, 0), (256, 1e-3, 0, 0)])
def test_propagation_writes_stay_inside_their_buffers(N, dx, colv, fused, monkeypatch):
    if N >= 512:
        _env(monkeypatch, TS_FFT_E=32, TS_COL_VARIANT=colv, TS_ROW_VARIANT=2, TS_PROP_STREAMS=1, TS_FUSED=fused)
    S, B = 3, 3
    plan = ts.Plan(LAM, N, dx, [62.5] * S, [1e-14] * S, l0=5e-3, L0=10.0, max_batch=B)
    ph = _phasors(plan, N, S)
    outs = _propagation_cases(plan, N, S, B, ph.t)
    assert all(g.margins_intact() for g in outs + [ph])
    assert np.isfinite(outs[0].t.cpu().numpy()).all()
    plan.close()


def test_split_bf16_writes_stay_inside_their_buffers():
    N, dx, S, B = 1024, 5e-4, 2, 3
    plan = ts.Plan(LAM, N, dx, [62.5] * S, [1e-14] * S, l0=5e-3, L0=10.0, max_batch=B, flags=ts.TS_PLAN_SPLIT_BF16)
    ph = _phasors(plan, N, S)
    outs = _propagation_cases(plan, N, S, B, ph.t)
    assert all(g.margins_intact() for g in outs + [ph])
    plan.close()


def test_regenerated_screens_and_field_groups_stay_inside(monkeypatch):
    # screens regenerated from the seed inside the call, on two concurrent field groups
    _env(monkeypatch, TS_PROP_STREAMS=2, TS_FUSED=0)
    N, dx, S, B = 1024, 5e-4, 3, 3
    plan = ts.Plan(LAM, N, dx, [62.5] * S, [1e-14] * S, l0=5e-3, L0=10.0, max_batch=B)
    plan.set_sources([0.01, 0.012, 0.014])
    U = Guarded((B, N, N), torch.complex64)
    plan.propagate(U.t, B, phi_group=1, flags=ts.TS_PROP_SOURCE, seed=11, real_base=5)
    G = Guarded((B, N, N), torch.complex64, _random_field(B, N, 5))
    plan.propagate_backward(G.t, B, phi_group=1, seed=11, real_base=5)
    torch.cuda.synchronize()
    plan.device_status()
    assert U.margins_intact() and G.margins_intact()
    plan.close()


@pytest.mark.parametrize("N", [256, 1024])
def test_screen_synthesis_writes_stay_inside(N):
    # independent screens (2 realizations, subharmonics) and three AR steps, every output guarded
    dx, S = 1e-3 if N == 256 else 5e-4, 3
    plan = ts.Plan(LAM, N, dx, [100.0] * S, [1e-14] * S, l0=5e-3, L0=10.0, sh_levels=3, max_batch=1)
    phi = Guarded((2, S, N, N), torch.float32)
    ph = Guarded((2, S, N, N), torch.complex64)
    plan.make_screens(phi.t, 21, real_base=1, n_real=2, phasor=ph.t)
    spec = Guarded((S, N, N), torch.complex64)
    sh = Guarded((S, 27), torch.complex128)
    phi1 = Guarded((S, N, N), torch.float32)
    ph1 = Guarded((S, N, N), torch.complex64)
    for t in range(3):
        plan.evolve_screens(spec.t, phi1.t, 21, t, 0.99, real=0, vx=1.0, vy=0.5, T=1e-3, sh_state=sh.t, phasor=ph1.t)
    torch.cuda.synchronize()
    plan.device_status()
    assert all(g.margins_intact() for g in (phi, ph, spec, sh, phi1, ph1))
    plan.close()


def test_moment_accumulators_stay_inside():
    N, dx, S, B = 128, 2e-3, 2, 6
    plan = ts.Plan(LAM, N, dx, [300.0] * S, [3e-14] * S, l0=5e-3, L0=10.0, max_batch=B)
    plan.set_sources([0.0, 0.03, 0.05])
    I = torch.zeros((B, N, N), dtype=torch.float32, device=DEV)
    U = torch.zeros((B, N, N), dtype=torch.complex64, device=DEV)
    mean = Guarded((3, N, N), torch.float64)
    m2 = Guarded((3, N, N), torch.float64)
    count = 0
    for c in range(2):
        plan.propagate(U, B, phi_group=3, flags=ts.TS_PROP_SOURCE | ts.TS_PROP_INTENSITY, seed=3, real_base=2 * c,
                       intensity=I)
        plan.moments_accumulate(I, B, 3, count, mean.t, m2.t)
        count += B // 3
    si_map = Guarded((3, N, N), torch.float64)
    si_mean = Guarded((3,), torch.float64)
    si_c = Guarded((3,), torch.float64)
    plan.moments_finalize(mean.t, m2.t, 3, count, si_map=si_map.t, si_mean=si_mean.t, si_center=si_c.t)
    torch.cuda.synchronize()
    plan.device_status()
    assert all(g.margins_intact() for g in (mean, m2, si_map, si_mean, si_c))
    plan.close()
