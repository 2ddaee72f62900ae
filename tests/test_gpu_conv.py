"""Tensor-core 3x3 convolution (hp_conv3x3_bf16) against the FP64 oracle
convolution on the same BF16-rounded inputs and weights.  Bar: |y_gpu - y| <=
2^-7 * max|y| per element (BF16 output rounding + FP32 accumulation)."""
import numpy as np
import pytest

from oracle import cnn as C

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
hp = pytest.importorskip("paper_2109_09363_gb300")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_09363_gb300 import build
    build.build()
    return torch.device("cuda:0")


@pytest.mark.parametrize("cin,cout", [(32, 32), (32, 64), (64, 32), (64, 64)])
@pytest.mark.parametrize("shape", [(1, 8, 16), (2, 37, 53), (1, 128, 128), (1, 20, 200), (2, 67, 256)])
def test_conv3x3_tensor_core_matches_oracle(dev, cin, cout, shape):
    B, H, W = shape
    rng = np.random.default_rng(cin * 7 + cout + H)
    x = torch.from_numpy(rng.standard_normal((B, H, W, cin)).astype(np.float32)).to(torch.bfloat16)
    w = torch.from_numpy((rng.standard_normal((3, 3, cout, cin)) / np.sqrt(9 * cin))
                         .astype(np.float32)).to(torch.bfloat16)
    bias = torch.from_numpy(rng.standard_normal(cout).astype(np.float32) * 0.1)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    for relu in (False, True):
        y = hp.hp_conv3x3_bf16(x.to(dev), w.to(dev), bias.to(dev), relu, err=err)
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        xf = x.float().numpy().astype(np.float64)
        wf = w.float().numpy().astype(np.float64)   # [dy][dx][co][ci]
        w_oihw = np.transpose(wf, (2, 3, 0, 1))
        for b in range(B):
            ref = C.conv3x3(np.transpose(xf[b], (2, 0, 1)), w_oihw, bias.numpy().astype(np.float64))
            if relu:
                ref = np.maximum(ref, 0.0)
            got = np.transpose(y[b].float().cpu().numpy(), (2, 0, 1))
            scale = np.abs(ref).max()
            assert np.abs(got - ref).max() <= 2.0 ** -7 * scale, (b, np.abs(got - ref).max(), scale)
