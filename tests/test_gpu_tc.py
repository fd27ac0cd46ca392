"""Split-BF16 tensor-core DFT (tcgen05): accuracy of the 32-point building block against numpy."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2604_07248_gb300 import binding as bd  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("sign", [-1, 1])
def test_tc_dft32_matches_fft(sign, layout):
    nvec = 300  # three CTAs, the last one ragged
    rng = np.random.default_rng(7)
    x = (rng.standard_normal((nvec, 32)) + 1j * rng.standard_normal((nvec, 32))).astype(np.complex64)
    xd = torch.from_numpy(x).to(DEV)
    Xd = torch.zeros_like(xd)
    err = bd.tc_dft32(xd, Xd, sign=sign, layout=layout)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    ref = np.fft.fft(x.astype(np.complex128), axis=1) if sign < 0 else np.fft.ifft(x.astype(np.complex128), axis=1) * 32
    got = Xd.cpu().numpy()
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    # hi.hi + hi.lo + lo.hi keeps about 16 bits per product; FP32 accumulation over 64 terms
    assert rel < 1e-4, rel
    assert rel > 1e-9  # the tensor-core path is really BF16-based (not an FP32 FFT)


def test_tc_mn_major_descriptor_reading():
    # the same MN-major data with the two descriptor strides exchanged is not a DFT: the stride
    # assignment used by the tensor-core passes is the one the hardware reads
    rng = np.random.default_rng(8)
    x = (rng.standard_normal((128, 32)) + 1j * rng.standard_normal((128, 32))).astype(np.complex64)
    xd = torch.from_numpy(x).to(DEV)
    Xd = torch.zeros_like(xd)
    err = bd.tc_dft32(xd, Xd, sign=-1, layout=2)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    ref = np.fft.fft(x.astype(np.complex128), axis=1)
    got = Xd.cpu().numpy()
    assert np.all(np.isfinite(got))  # the operand window is zeroed before staging
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) > 0.1
