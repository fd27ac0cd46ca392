"""D2NN training loop (Sec. 2.5) on the GPU against the oracle: the Adam kernel, and whole epochs
(propagation through a fresh realization of a planned HV5/7 path, two-mask receiver, loss, receiver
adjoint, Adam with the one-cycle learning rate)."""
import numpy as np
import pytest

import oracle as O
from oracle import training as OT

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2604_07248_gb300 import binding as bd  # noqa: E402
from paper_2604_07248_gb300 import training as tr  # noqa: E402

DEV = torch.device("cuda:0")


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def test_adam_kernel_matches_oracle():
    rng = np.random.default_rng(5)
    n = 100003  # ragged against the 256-thread blocks
    p0 = rng.standard_normal(n).astype(np.float32)
    p, m, v = torch.from_numpy(p0).to(DEV), torch.zeros(n, device=DEV), torch.zeros(n, device=DEV)
    po, mo, vo = p0.astype(np.float64), np.zeros(n), np.zeros(n)
    for t in range(1, 4):
        g0 = rng.standard_normal(n).astype(np.float32)
        bd.adam_step(p, torch.from_numpy(g0).to(DEV), m, v, t, lr=0.01)
        po, mo, vo = OT.adam(po, g0.astype(np.float64), mo, vo, t, lr=0.01)
    torch.cuda.synchronize()
    assert rel_l2(p.cpu().numpy(), po) < 1e-6
    assert rel_l2(m.cpu().numpy(), mo) < 1e-6
    assert rel_l2(v.cpu().numpy(), vo) < 1e-6


def test_three_training_epochs_match_oracle():
    # the paper's set-up scaled to N = 256 (dx = 1.36 mm, same 0.35 m grid): 1064 nm, 4.5 mm waist,
    # 1500 m HV5/7 path at sigma_R^2 = 0.2 placed by the planner, 12-inch aperture.  Squared-error
    # loss (smooth), normalised to the free-space peak, and seeded N(0, 0.1) starting masks: at zero
    # phase the first mask's gradient vanishes exactly (the receiver is then the identity), which
    # leaves nothing to compare.  The mask updates (not the masks) are compared.
    lam, N, dx, w0, ap, seed, epochs = 1.064e-6, 256, 1.36e-3, 4.5e-3, 0.3048, 2604, 20000
    A, h, cn2p, dz, cn2 = tr.hv57_path(lam, 1500.0, 0.2, N, dx, 0.1)
    rng = np.random.default_rng(7)
    th0 = [rng.normal(0, 0.1, (N, N)).astype(np.float32) for _ in range(2)]
    trainer = tr.D2nnTrainer(lam, N, dx, list(dz), list(cn2), w0, ap, seed, epochs, l0=5e-3, L0=10.0, device=DEV,
                             loss_kind=1, init_masks=th0)
    losses = []
    for e in range(3):
        trainer.epoch(e)
        torch.cuda.synchronize()
        losses.append(trainer.loss.item())
    md = O.medium(lam, N, dx, l0=5e-3, L0=10.0)
    Aap = O.aperture(N, dx, ap)
    src = O.source_gaussian(N, dx, w0)
    Uvac = O.propagate(md, list(dz), None, src)
    Iref = np.abs(Aap * Uvac) ** 2
    assert rel_l2(trainer.Iref.cpu().numpy(), Iref) < 1e-5
    scale = 1.0 / Iref.max() ** 2
    assert abs(trainer.loss_scale / scale - 1) < 1e-5
    th1, th2 = th0[0].astype(np.float64), th0[1].astype(np.float64)
    state = tuple(np.zeros((N, N)) for _ in range(4))
    for e in range(3):
        lr = OT.one_cycle(e, epochs, 0.01)
        loss, th1, th2, state = OT.epoch(O, md, list(dz), list(cn2), seed, e, src, Aap, th1, th2, Iref, state, e + 1,
                                         lr, kind=1, scale=scale)
        assert abs(losses[e] / loss - 1) < 1e-4, (e, losses[e], loss)
    d1 = trainer.th[0].cpu().numpy().astype(np.float64) - th0[0]
    d2 = trainer.th[1].cpu().numpy().astype(np.float64) - th0[1]
    assert rel_l2(d1, th1 - th0[0]) < 2e-3
    assert rel_l2(d2, th2 - th0[1]) < 2e-3
    # the normalised loss puts the gradients above Adam's eps: where the beam is, the masks move by
    # sign-like steps of about lr per epoch
    lr_sum = sum(OT.one_cycle(e, epochs, 0.01) for e in range(3))
    assert np.abs(th1 - th0[0]).max() > 0.5 * lr_sum
    assert np.abs(th2 - th0[1]).max() > 0.5 * lr_sum
