"""The SmallScale network (Sec. 3.1: the MultiScale with fewer filters, every
64-channel layer at 32 channels), the MonoScale (one feed-forward branch of
nine convolutions at full resolution) and the Unet (five scales, max pooling,
concatenated skip features) on the GPU against the FP64 oracle:
1. the forward (hp_cnn_forward), under the bar of the MultiScale forward test;
2. the hybrid projection from the same guess;
3. the training gradient (hand-written backward: on the tensor cores from a
   width of 32 pixels, on CUDA cores below) against the oracle backward,
   under the bar of the MultiScale gradient tests;
4. a few Adam steps lower the loss;
5. the architecture is kept and checked (parameter counts of the other
   architecture are rejected)."""
import numpy as np
import pytest

import oracle
from oracle import cnn as C
from oracle import train as TR
from paper_2109_09363_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
hp = pytest.importorskip("paper_2109_09363_gb300")

ARCHS = ["smallscale", "monoscale", "unet"]   # forward, hybrid projection and training
FORWARD_ARCHS = ARCHS


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_09363_gb300 import build
    build.build()
    oracle.build()
    return torch.device("cuda:0")


def random_params(seed, arch):
    rng = np.random.default_rng(seed)
    return [(w, 0.05 * rng.standard_normal(b.shape)) for w, b in C.init_params(seed, arch)]


def bf16_weights(params):
    return [(C.round_bf16(w), b.astype(np.float32).astype(np.float64)) for w, b in params]


def case(B, n, seed):
    us, vs, fs = [], [], []
    for b in range(B):
        u, v = W.vortex_velocity(n, n, 40 + seed + b, n_vortices=8, width=(n / 32, n / 8))
        fs.append(W.random_obstacles(n, n, 50 + seed + b, rect_side=(n / 16, n / 4),
                                     disc_radius=(n / 32, n / 8)))
        us.append(u); vs.append(v)
    return (np.stack(us).astype(np.float32), np.stack(vs).astype(np.float32), np.stack(fs))


@pytest.mark.parametrize("arch", FORWARD_ARCHS)
@pytest.mark.parametrize("B,n", [(2, 64), (1, 128), (3, 32), (2, 16)])
def test_network_forward_matches_oracle(dev, arch, B, n):
    params = random_params(3, arch)
    u, v, fl = case(B, n, 1)
    cnn = hp.CNN(B, n, n, params=C.flatten(params), arch=arch)
    assert cnn.arch == arch and cnn.n_params == C.param_count(arch)
    assert hp.load_library().hp_cnn_get_arch(cnn.handle) == hp.CNN_ARCHS[arch]
    ud, vd, fd = (torch.from_numpy(a).to(dev) for a in (u, v, fl))
    div = hp.hp_divergence(ud, vd, fd)
    phi_hat, s = hp.hp_cnn_forward(cnn, div, fd)
    torch.cuda.synchronize()
    cnn.check()
    pw = bf16_weights(params)
    for b in range(B):
        d = div[b].cpu().numpy().astype(np.float64)
        sb = float(s[b].cpu())
        ref = C.forward(pw, d / sb, fl[b], act_round=C.round_bf16)
        got = phi_hat[b].cpu().numpy()
        assert np.abs(got - ref).max() <= 2e-2 * np.abs(ref).max(), np.abs(got - ref).max()


# E_k of FP32 sweeps from a guess of magnitude |phi| carries an error of some
# tens of 2^-24 * mean|phi| (up to 94 on these cases over 3,000 sweeps, with
# an FP32 emulation of the kernel's operation order): the rough guesses of
# untrained networks (|phi| ~ 0.3 against E ~ 1e-3) make that a few 1e-4 of E
# near the threshold, so the stop may move by a sweep or two
E_ULPS = 256


@pytest.mark.parametrize("arch", FORWARD_ARCHS)
def test_hybrid_projection_matches_oracle_from_the_same_guess(dev, arch):
    """The GPU stops where its own E history first reaches E_t; that history
    tracks the oracle's (same guess, same sweeps) within the FP32 bound above;
    the velocity equals the oracle's run to the GPU's count."""
    B, n, thr, cap = 2, 64, 1e-3, 3000
    params = random_params(5, arch)
    u, v, fl = case(B, n, 7)
    cnn = hp.CNN(B, n, n, params=C.flatten(params), arch=arch)
    ctx = hp.Context(B, n, n)
    ud, vd, fd = (torch.from_numpy(a).to(dev) for a in (u, v, fl))
    div = hp.hp_divergence(ud, vd, fd)
    phi_hat, s = hp.hp_cnn_forward(cnn, div, fd)
    phi0 = (phi_hat.cpu().numpy() * s.cpu().numpy()[:, None, None]).astype(np.float64)
    out = hp.hp_project_hybrid(ctx, cnn, ud, vd, fd, hp.ProjectParams(threshold=thr, max_iters=cap),
                               hist_len=cap + 2)
    torch.cuda.synchronize()
    u64, v64 = u.astype(np.float64), v.astype(np.float64)
    gi = out["iters"].cpu().numpy()
    gh = out["e_hist"].cpu().numpy()
    gc = out["converged"].cpu().numpy()
    for b in range(B):
        kg = int(gi[b])
        assert np.all(gh[b, :kg] > thr)
        assert (gh[b, kg] <= thr) == bool(gc[b]) and (gc[b] or kg == cap)
        # the oracle run to exactly the GPU's count (threshold 0: the cap stops
        # it), with its E history
        one = oracle.project(u64[b], v64[b], fl[b], 0.0, kg, phi0=phi0[b], hist_len=kg + 1)
        eo = one["e_hist"][0][:kg + 1]
        bound = E_ULPS * 2.0 ** -24 * np.abs(one["phi"][0]).mean()
        dev_e = np.abs(gh[b, :kg + 1] - eo)
        assert np.all(dev_e <= bound), (b, dev_e.max(), bound)
        umax = np.abs(one["u"][0]).max()
        assert np.abs(ud.cpu().numpy()[b] - one["u"][0]).max() <= 1e-5 * umax


def oracle_gradient(params, phi_gpu, div, fl, tgt, s, lam, act_round):
    B = div.shape[0]
    pw = bf16_weights(params)
    total = [(np.zeros_like(w), np.zeros_like(b)) for w, b in pw]
    L = 0.0
    for b in range(B):
        d = div[b].astype(np.float64)
        _, tape = C.forward(pw, d / s[b], fl[b], keep=True, act_round=act_round)
        lb, gphi = TR.loss_and_grad(phi_gpu[b], tgt[b], d, fl[b], s[b], lam)
        L += lb / B
        gr = C.backward(pw, tape, gphi / B)
        total = [(tw + gw, tb + gb) for (tw, tb), (gw, gb) in zip(total, gr)]
    return L, total


@pytest.mark.parametrize("arch,B,ny,nx", [
    (a, *shape) for a in ARCHS
    for shape in [(2, 16, 16), (2, 32, 32), (2, 128, 128), (1, 64, 160)]] + [
    ("unet", 1, 256, 512)])
def test_network_gradient_matches_oracle_backward(dev, arch, B, ny, nx):
    """16 x 16: every branch on CUDA cores; 32 x 32: the SmallScale's coarse
    branches (8 and 16 pixels wide) on CUDA cores, full resolution on the
    tensor cores; the larger sizes on the tensor cores throughout (160 = a
    full and a partial 128-pixel segment).  The Unet's levels narrower than
    32 pixels (down to 1 x 1 at 16 x 16) run on CUDA cores, with the
    concatenation and pooling transposes between BF16 and FP32 levels;
    256 x 512 puts levels 0-3 on the tensor cores."""
    rng = np.random.default_rng(B + nx + 1)
    params = random_params(13, arch)
    u, v, fl = W.training_case(1, max(ny, nx), 710)
    u, v, fl = u[:, :ny, :nx + 1], v[:, :ny + 1, :nx], fl[:, :ny, :nx]
    u, v, fl = np.repeat(u, B, 0), np.repeat(v, B, 0), np.ascontiguousarray(np.repeat(fl, B, 0))
    if B > 1:
        u[1] = np.roll(u[1], 11, axis=1)
        v[1] = np.roll(v[1], 7, axis=0)
    ud = torch.from_numpy(np.ascontiguousarray(u, np.float32)).to(dev)
    vd = torch.from_numpy(np.ascontiguousarray(v, np.float32)).to(dev)
    fd = torch.from_numpy(fl).to(dev)
    div = hp.hp_divergence(ud, vd, fd)
    tgt = torch.from_numpy(rng.standard_normal((B, ny, nx)).astype(np.float32)).to(dev)
    cnn = hp.CNN(B, ny, nx, params=C.flatten(params), arch=arch)
    tr = hp.Trainer(cnn, B, ny, nx)
    lam = 1.0
    g, loss = tr.gradient(div, fd, tgt, lambda_div=lam)
    assert g.numel() == C.param_count(arch)
    phi_gpu, s = hp.hp_cnn_forward(cnn, div, fd)
    torch.cuda.synchronize()
    cnn.check()
    args = (phi_gpu.cpu().numpy(), div.cpu().numpy(), fl, tgt.cpu().numpy(),
            [float(x) for x in s.cpu()], lam)
    L, ref = oracle_gradient(params, *args, act_round=C.round_bf16)
    assert np.isclose(float(loss.item()), L, rtol=1e-4)
    _, ref64 = oracle_gradient(params, *args, act_round=None)
    flat = g.cpu().numpy()
    k = 0
    for (w, b), (w64, b64) in zip(ref, ref64):
        nw, nb = w.size, b.size
        gw, gb = flat[k:k + nw], flat[k + nw:k + nw + nb]
        scale = max(np.abs(w).max(), np.abs(b).max())
        sens = max(np.abs(w - w64).max(), np.abs(b - b64).max())
        bar = max(5e-2 * scale, 3.0 * sens) + 1e-9
        assert np.abs(gw - w.ravel()).max() <= bar, (k, np.abs(gw - w.ravel()).max(), scale, sens)
        assert np.abs(gb - b.ravel()).max() <= bar, (k, np.abs(gb - b.ravel()).max(), scale)
        k += nw + nb
    assert k == flat.size


@pytest.mark.parametrize("arch", ARCHS)
def test_adam_steps_lower_the_loss(dev, arch):
    B, n = 8, 64
    rng = np.random.default_rng(21)
    u, v, fl = W.training_case(B, n, 720)
    ud = torch.from_numpy(u.astype(np.float32)).to(dev)
    vd = torch.from_numpy(v.astype(np.float32)).to(dev)
    fd = torch.from_numpy(fl).to(dev)
    div = hp.hp_divergence(ud, vd, fd)
    tgt = torch.from_numpy(rng.standard_normal((B, n, n)).astype(np.float32)).to(dev)
    from paper_2109_09363_gb300 import training as T
    cnn = hp.CNN(B, n, n, params=T.init_params(seed=2, arch=arch), arch=arch)
    tr = hp.Trainer(cnn, B, n, n)
    losses = [float(tr.step(div, fd, tgt, lr=1e-3, lambda_div=0.0).item()) for _ in range(30)]
    assert all(np.isfinite(losses))
    assert losses[-1] < losses[0], (losses[0], losses[-1])
    tr.sync_params()
    p = cnn.get_params()
    assert p.size == C.param_count(arch) and np.all(np.isfinite(p))


@pytest.mark.parametrize("arch", ARCHS)
def test_parameter_counts_are_checked(dev, arch):
    B, n = 1, 32
    cnn = hp.CNN(B, n, n, arch=arch)
    with pytest.raises(hp.HprojError):
        cnn.set_params(C.flatten(C.init_params(1)))  # MultiScale-sized vector
    with pytest.raises(ValueError):
        hp.CNN(B, n, n, arch="resnet")


def test_unet_at_the_tensor_core_widths_and_argument_checks(dev):
    """512 x 256: every level from 32 pixels wide up on the tensor cores, the
    n/16 bottom (32 x 16) on the gather kernel; the Unet and its trainer want
    sizes that are multiples of 16."""
    B, ny, nx = 1, 256, 512
    params = random_params(9, "unet")
    u, v = W.vortex_velocity(ny, nx, 61, n_vortices=12, width=(4, 24))
    fl = W.random_obstacles(ny, nx, 62, rect_side=(16, 64), disc_radius=(8, 32))
    ud = torch.from_numpy(u[None].astype(np.float32)).to(dev)
    vd = torch.from_numpy(v[None].astype(np.float32)).to(dev)
    fd = torch.from_numpy(fl[None]).to(dev)
    cnn = hp.CNN(B, ny, nx, params=C.flatten(params), arch="unet")
    div = hp.hp_divergence(ud, vd, fd)
    phi_hat, s = hp.hp_cnn_forward(cnn, div, fd)
    torch.cuda.synchronize()
    cnn.check()
    d = div[0].cpu().numpy().astype(np.float64)
    ref = C.forward(bf16_weights(params), d / float(s[0].cpu()), fl, act_round=C.round_bf16)
    got = phi_hat[0].cpu().numpy()
    assert np.abs(got - ref).max() <= 2e-2 * np.abs(ref).max(), np.abs(got - ref).max()
    with pytest.raises(hp.HprojError):
        hp.CNN(1, 40, 48, arch="unet")
    with pytest.raises(hp.HprojError):
        hp.Trainer(cnn, B, 40, 48)
