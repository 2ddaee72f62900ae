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


@pytest.mark.parametrize("cin,cout,shape", [(64, 64, (8, 512, 512)), (32, 64, (16, 256, 256)),
                                            (64, 32, (2, 300, 640)), (32, 32, (4, 129, 330))])
def test_conv3x3_full_size_sampled(dev, cin, cout, shape):
    """Sizes at which every persistent CTA walks several work items and the
    input-row ring wraps inside an item; the oracle evaluates sampled output
    pixels one by one (all four borders, corners and random interior)."""
    B, H, W = shape
    g = torch.Generator(device="cpu").manual_seed(cin + cout + H)
    x = torch.randn((B, H, W, cin), generator=g).to(torch.bfloat16)
    w = (torch.randn((3, 3, cout, cin), generator=g) / (3 * cin ** 0.5)).to(torch.bfloat16)
    bias = torch.randn(cout, generator=g) * 0.1
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    y = hp.hp_conv3x3_bf16(x.to(dev), w.to(dev), bias.to(dev), True, err=err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    y = y.float().cpu().numpy()
    xf = x.float().numpy().astype(np.float64)
    w_oihw = np.transpose(w.float().numpy().astype(np.float64), (2, 3, 0, 1))
    bf = bias.numpy().astype(np.float64)
    rng = np.random.default_rng(H + W)
    pts = [(b, i, j) for b in range(B) for i in (0, H - 1) for j in (0, W - 1)]
    for b in range(B):
        for i in rng.integers(0, H, 24):
            pts += [(b, int(i), 0), (b, int(i), W - 1), (b, int(i), int(rng.integers(0, W)))]
        for j in rng.integers(0, W, 24):
            pts += [(b, 0, int(j)), (b, H - 1, int(j))]
        pts += [(b, int(i), int(j)) for i, j in zip(rng.integers(0, H, 200),
                                                     rng.integers(0, W, 200))]
    worst, scale = 0.0, 0.0
    for b, i, j in pts:
        rows = np.clip([i - 1, i, i + 1], 0, H - 1)
        cols = np.clip([j - 1, j, j + 1], 0, W - 1)
        patch = np.transpose(xf[b][np.ix_(rows, cols)], (2, 0, 1))   # [cin][3][3]
        ref = np.maximum(C.conv3x3(patch, w_oihw, bf)[:, 1, 1], 0.0)
        worst = max(worst, float(np.abs(y[b, i, j] - ref).max()))
        scale = max(scale, float(np.abs(ref).max()))
    assert worst <= 2.0 ** -7 * scale, (worst, scale)
