"""The allocation-free norm entry point (hp_div_norms_noalloc) against the
context-based hp_div_norms, through the C ABI.

Some callers cannot allocate device memory (a framework that owns all device
memory through its own pool, a latency-critical loop); hp_div_norms_noalloc
serves them with a fixed scratch array inside the library.  This file is
collected last so that a run stopping at its first failure has already run
every other test; it also passes alone in a fresh process."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
hp = pytest.importorskip("paper_2109_09363_gb300")

RTOL = 1e-5  # the tolerance of the context-based norm test


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_09363_gb300 import build
    build.build()
    return torch.device("cuda:0")


def fields(B, ny, nx, seed):
    rng = np.random.default_rng(seed)
    u = torch.from_numpy(rng.standard_normal((B, ny, nx + 1)).astype(np.float32))
    v = torch.from_numpy(rng.standard_normal((B, ny + 1, nx)).astype(np.float32))
    fl = torch.from_numpy((rng.random((B, ny, nx)) < 0.15).astype(np.uint8))
    return u, v, fl


def test_noalloc_norms_match_context_norms_on_consecutive_calls(dev):
    cases = [(4, 130, 300, 1), (2, 37, 1000, 2)]
    ctx = hp.Context(4, 130, 1000)
    for B, ny, nx, seed in cases + cases:
        u, v, fl = (t.to(dev) for t in fields(B, ny, nx, seed))
        e1_ref, einf_ref = hp.hp_div_norms(ctx, u, v, fl)
        e1_out = torch.empty(B, dtype=torch.float64, device=dev)
        einf_out = torch.empty(B, dtype=torch.float64, device=dev)
        for _ in range(2):
            e1_out.fill_(-1.0)
            einf_out.fill_(-1.0)
            hp.hp_div_norms_noalloc(u, v, fl, e1_out, einf_out)
            torch.cuda.synchronize()
            assert np.allclose(e1_out.cpu().numpy(), e1_ref.cpu().numpy(), rtol=RTOL, atol=0)
            assert np.allclose(einf_out.cpu().numpy(), einf_ref.cpu().numpy(), rtol=RTOL, atol=0)


def test_noalloc_allocates_no_device_memory(dev):
    # after a first call (which sets up the scratch address of this context),
    # two calls with preallocated outputs leave the device's free memory as
    # it was: neither the library nor torch allocates
    B, ny, nx = 4, 130, 300
    u, v, fl = (t.to(dev) for t in fields(B, ny, nx, 5))
    e1_out = torch.empty(B, dtype=torch.float64, device=dev)
    einf_out = torch.empty(B, dtype=torch.float64, device=dev)
    hp.hp_div_norms_noalloc(u, v, fl, e1_out, einf_out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    stats0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    for _ in range(2):
        hp.hp_div_norms_noalloc(u, v, fl, e1_out, einf_out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    stats1 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    assert free1 == free0
    assert stats1 == stats0


def test_noalloc_at_its_largest_shape(dev):
    # 16 x 2048 x 2048 uses every partial-sum slot of the scratch array
    B, ny, nx = 16, 2048, 2048
    assert B * ny * ((nx + 255) // 256) == 262144
    g = torch.Generator(device=dev).manual_seed(11)
    u = torch.randn((B, ny, nx + 1), generator=g, device=dev)
    v = torch.randn((B, ny + 1, nx), generator=g, device=dev)
    fl = (torch.rand((B, ny, nx), generator=g, device=dev) < 0.15).to(torch.uint8)
    ctx = hp.Context(B, ny, nx)
    e1_ref, einf_ref = hp.hp_div_norms(ctx, u, v, fl)
    for _ in range(2):
        e1, einf = hp.hp_div_norms_noalloc(u, v, fl)
        torch.cuda.synchronize()
        assert np.allclose(e1.cpu().numpy(), e1_ref.cpu().numpy(), rtol=RTOL, atol=0)
        assert np.allclose(einf.cpu().numpy(), einf_ref.cpu().numpy(), rtol=RTOL, atol=0)
    ctx.close()


@pytest.mark.parametrize("B,ny,nx", [(16385, 1, 1), (1, 262145, 1), (1, 70000, 1)])
def test_noalloc_rejects_shapes_beyond_its_scratch(dev, B, ny, nx):
    # more grids than its batch limit, more 256-cell blocks than partials, or
    # more rows than one CUDA grid dimension covers
    u = torch.zeros((B, ny, nx + 1), dtype=torch.float32, device=dev)
    v = torch.zeros((B, ny + 1, nx), dtype=torch.float32, device=dev)
    fl = torch.zeros((B, ny, nx), dtype=torch.uint8, device=dev)
    with pytest.raises(hp.HprojError):
        hp.hp_div_norms_noalloc(u, v, fl)
