"""Split-precision DFTs on the tensor cores (tcgen05.mma, FP32 accumulation)
against the FP64 transform of the oracle (numpy's FFT of the same data)."""
import numpy as np
import pytest

from tests import _gpu

pytestmark = pytest.mark.gpu
# hi+lo split: BF16 pairs keep ~16 significant bits, FP16 pairs ~22
TOL = {"bf16x3": 2e-5, "fp16x3": 2e-6}


@pytest.fixture(scope="module")
def torch():
    return _gpu.torch_cuda()


@pytest.mark.parametrize("precision", ["bf16x3", "fp16x3"])
@pytest.mark.parametrize("sign", [-1, 1])
@pytest.mark.parametrize("nvec,scale", [(200, 1.0), (64, 3e3), (7, 1e-3)])
def test_dft64_on_tensor_cores(torch, precision, sign, nvec, scale):
    from paper_1904_09409_gb300 import funnel as f
    rng = np.random.default_rng(nvec)
    x = (rng.standard_normal((nvec, 64)) + 1j * rng.standard_normal((nvec, 64))) * scale
    xd = torch.from_numpy(x.astype(np.complex64)).cuda()
    yd = torch.empty_like(xd)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    f.ft_tc_dft64(xd, yd, sign, precision, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    x32 = x.astype(np.complex64).astype(np.complex128)
    ref = np.fft.fft(x32, axis=1) if sign < 0 else 64 * np.fft.ifft(x32, axis=1)
    got = yd.cpu().numpy().astype(np.complex128)
    e = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert e <= TOL[precision], (precision, e)
