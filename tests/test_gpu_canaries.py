"""Out-of-bounds writes, checked without a memory checker:

- every caller-owned output is a view into a larger buffer whose margins
  hold a canary pattern; after the call the margins must be unchanged (no
  write before or past the array), on ragged multi-tile shapes;
- read-only inputs must be unchanged;
- the library's own workspaces (context, network, trainer) carry guard zones
  that hp_ctx_check / hp_cnn_check / hp_trainer_check compare after the
  calls, at and below each object's largest shape."""
import numpy as np
import pytest

from paper_2109_09363_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
hp = pytest.importorskip("paper_2109_09363_gb300")

PAD = 64  # elements on each side: keeps 16-byte alignment for every dtype here
CANARY = {torch.float32: 12345.678, torch.float64: -7.25e300, torch.int32: 0x5A5A5A5A,
          torch.uint8: 0xA5, torch.bfloat16: -3.5}


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_09363_gb300 import build
    build.build()
    return torch.device("cuda:0")


class Padded:
    """A contiguous tensor of `shape` inside a canary-filled buffer."""

    def __init__(self, shape, dtype, dev, init=None):
        n = int(np.prod(shape))
        self.n = n
        self.base = torch.full((n + 2 * PAD,), CANARY[dtype], dtype=dtype, device=dev)
        self.t = self.base[PAD:PAD + n].view(shape)
        if init is not None:
            self.t.copy_(init)

    def margins_intact(self):
        torch.cuda.synchronize()
        c = torch.full((PAD,), CANARY[self.base.dtype], dtype=self.base.dtype,
                       device=self.base.device)
        return torch.equal(self.base[:PAD], c) and torch.equal(self.base[PAD + self.n:], c)


def fields(B, ny, nx, seed):
    us, vs, fs = [], [], []
    for b in range(B):
        u, v = W.vortex_velocity(ny, nx, 500 + seed + b, n_vortices=6, width=(2.0, 10.0))
        us.append(u); vs.append(v)
        fs.append(W.random_obstacles(ny, nx, 600 + seed + b, rect_side=(4, 20),
                                     disc_radius=(3, 10)))
    return (torch.from_numpy(np.stack(us).astype(np.float32)),
            torch.from_numpy(np.stack(vs).astype(np.float32)),
            torch.from_numpy(np.stack(fs)))


def out_dict(B, ny, nx, dev, hist=0):
    o = {"p": Padded((B, ny, nx), torch.float32, dev), "iters": Padded((B,), torch.int32, dev),
         "e1": Padded((B,), torch.float64, dev), "einf": Padded((B,), torch.float64, dev),
         "converged": Padded((B,), torch.uint8, dev)}
    if hist:
        o["e_hist"] = Padded((B, hist), torch.float64, dev)
    return o


@pytest.mark.parametrize("B,ny,nx", [(3, 67, 130), (1, 129, 257), (2, 5, 3), (2, 37, 264)])
def test_projection_path_writes_only_its_outputs(dev, B, ny, nx):
    u0, v0, f0 = fields(B, ny, nx, ny + nx)
    ctx = hp.Context(B, ny, nx)
    fl = f0.to(dev)
    fl_keep = fl.clone()
    for kernel in (0, 1, 2, 3):
        for bc in (dict(), dict(open_top=1, inflow=(nx // 3, 2 * nx // 3))):
            u = Padded(u0.shape, torch.float32, dev, u0)
            v = Padded(v0.shape, torch.float32, dev, v0)
            o = out_dict(B, ny, nx, dev, hist=40)
            prm = hp.ProjectParams(threshold=1e-4, max_iters=300, sweep_kernel=kernel, **bc)
            hp.hp_project(ctx, u.t, v.t, fl, prm, hist_len=40,
                          out={k: x.t for k, x in o.items()})
            for x in [u, v, *o.values()]:
                assert x.margins_intact(), (kernel, bc)
    div = Padded((B, ny, nx), torch.float32, dev)
    mask = Padded((B, ny, nx), torch.uint8, dev)
    hp.hp_divergence(u0.to(dev), v0.to(dev), fl, div_out=div.t)
    hp.hp_face_mask(fl, mask_out=mask.t)
    phi = Padded((B, ny, nx), torch.float32, dev)
    tgt = Padded((B, ny, nx), torch.float32, dev)
    div_keep = div.t.clone()
    hp.hp_jacobi_sweeps(ctx, torch.zeros_like(div.t), div.t, fl, 17, phi_out=phi.t)
    hp.hp_jacobi_target(ctx, div.t, fl, 23, target_out=tgt.t)
    e1 = Padded((B,), torch.float64, dev)
    einf = Padded((B,), torch.float64, dev)
    hp.hp_div_norms_noalloc(u0.to(dev), v0.to(dev), fl, e1.t, einf.t)
    rho = torch.ones((B, ny, nx), dtype=torch.float32, device=dev)
    uo = Padded(u0.shape, torch.float32, dev)
    vo = Padded(v0.shape, torch.float32, dev)
    ro = Padded((B, ny, nx), torch.float32, dev)
    for scheme in (0, 1):
        pp = hp.PlumeParams(inlet_x0=1, inlet_x1=nx - 1, scheme=scheme, u_in=0.1, open_top=1)
        hp.hp_advect_step(u0.to(dev), v0.to(dev), rho, fl, pp, uo.t, vo.t, ro.t)
    head = Padded((B, 3), torch.int32, dev)
    hp.hp_plume_head(ro.t, out=head.t)
    for x in (div, mask, phi, tgt, e1, einf, uo, vo, ro, head):
        assert x.margins_intact()
    assert torch.equal(fl, fl_keep) and torch.equal(div.t, div_keep)
    ctx.check()


@pytest.mark.parametrize("arch", ["multiscale", "unet"])
def test_network_path_writes_only_its_outputs(dev, arch):
    B, ny, nx = (2, 68, 132) if arch == "multiscale" else (2, 64, 144)
    u0, v0, f0 = fields(B, ny, nx, 7)
    from paper_2109_09363_gb300 import training as T
    cnn = hp.CNN(B, ny, nx, params=T.init_params(seed=3, arch=arch), arch=arch)
    ctx = hp.Context(B, ny, nx)
    fl = f0.to(dev)
    div = hp.hp_divergence(u0.to(dev), v0.to(dev), fl)
    ph = Padded((B, ny, nx), torch.float32, dev)
    s = Padded((B,), torch.float32, dev)
    hp.hp_cnn_forward(cnn, div, fl, phi_hat=ph.t, s_out=s.t)
    u = Padded(u0.shape, torch.float32, dev, u0)
    v = Padded(v0.shape, torch.float32, dev, v0)
    o = out_dict(B, ny, nx, dev)
    hp.hp_project_hybrid(ctx, cnn, u.t, v.t, fl, hp.ProjectParams(threshold=1e-4, max_iters=200),
                         out={k: x.t for k, x in o.items()})
    for x in [ph, s, u, v, *o.values()]:
        assert x.margins_intact()
    # a smaller batch and grid than the objects' largest
    hp.hp_cnn_forward(cnn, div[:1].contiguous(), fl[:1].contiguous())
    tr = hp.Trainer(cnn, B, ny, nx)
    tgt = torch.randn((B, ny, nx), device=dev)
    for _ in range(2):
        tr.step(div, fl, tgt, lambda_div=1.0)
    tr.pdnn_step(div, fl, torch.full((B,), 0.5, device=dev), norm=1)
    tr.check()
    ctx.check()
    assert cnn.check() == 0


@pytest.mark.parametrize("cin,cout,B,H,W", [(64, 32, 2, 33, 130), (32, 64, 1, 7, 29),
                                            (64, 64, 3, 16, 257)])
def test_convolution_writes_only_its_output(dev, cin, cout, B, H, W):
    g = torch.Generator(device=dev).manual_seed(cin + W)
    x = torch.randn((B, H, W, cin), generator=g, device=dev).to(torch.bfloat16)
    w = (0.1 * torch.randn((3, 3, cout, cin), generator=g, device=dev)).to(torch.bfloat16)
    bias = torch.randn(cout, generator=g, device=dev)
    y = Padded((B, H, W, cout), torch.bfloat16, dev)
    hp.hp_conv3x3_bf16(x, w, bias, True, y=y.t)
    assert y.margins_intact()
