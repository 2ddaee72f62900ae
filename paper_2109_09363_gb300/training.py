"""Training pairs from the plain solver and the training loop of the
MultiScale CNN; thin orchestration of the C ABI (every step runs in the
library's kernels)."""
from __future__ import annotations

import numpy as np
import torch

import paper_2109_09363_gb300 as hp
from paper_2109_09363_gb300 import workloads as W


# (cin, cout) of the 19 convolutions in network order: scale 1/4, 1/2, 1
LAYERS = ([(2, 32), (32, 64), (64, 64), (64, 32), (32, 1)] +
          2 * [(3, 32), (32, 64), (64, 64), (64, 64), (64, 64), (64, 32), (32, 1)])
# the SmallScale: every 64-channel layer at 32 channels
SMALL_LAYERS = ([(2, 32), (32, 32), (32, 32), (32, 32), (32, 1)] +
                2 * [(3, 32), (32, 32), (32, 32), (32, 32), (32, 32), (32, 32), (32, 1)])
# the MonoScale: one full-resolution branch of nine convolutions
MONO_LAYERS = [(2, 32), (32, 64)] + 5 * [(64, 64)] + [(64, 32), (32, 1)]
# the Unet: (cin, cout, kernel size), the last layer 1 x 1
UNET_LAYERS = ([(2, 32), (32, 32)] + 3 * [(32, 64), (64, 32)] + [(32, 64), (64, 64), (64, 32)]
               + 3 * [(64, 64), (64, 32)] + [(64, 32), (32, 32), (32, 1, 1)])
ARCH_LAYERS = {"multiscale": LAYERS, "smallscale": SMALL_LAYERS, "monoscale": MONO_LAYERS,
               "unet": UNET_LAYERS}


def init_params(seed: int = 0, arch: str = "multiscale") -> np.ndarray:
    """Initial parameters in the network's flat order (per layer weights
    [cout][cin][3][3] He-uniform, then zero biases), FP32."""
    g = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for layer in ARCH_LAYERS[arch]:
        cin, cout = layer[:2]
        taps = layer[2] ** 2 if len(layer) > 2 else 9
        lim = np.sqrt(6.0 / (taps * cin))
        parts.append(g.uniform(-lim, lim, taps * cin * cout))
        parts.append(np.zeros(cout))
    return np.concatenate(parts).astype(np.float32)


def generate_pairs(count: int, n: int, seed0: int = 0, sweeps: int = 40000,
                   chunk: int = 1024, device=None):
    """(div, flags, target) on the device: div of a seeded velocity field with
    obstacles, target = the scaled pressure phi of the plain solver after a
    fixed number of Jacobi sweeps from zero, as the mean of that iterate and
    one more sweep (this cancels the period-2 component that plain Jacobi
    never damps).

    The sweep count sets how much of the smooth part of phi the target holds:
    at 128^2, 8,000 sweeps leave 20-30 % relative L2 error against the exact
    solve, 30,000 about 1 %, 60,000 below 0.1 %; the error falls with
    sweeps / n^2."""
    dev = device or torch.device("cuda", torch.cuda.current_device())
    divs, fls, tgts = [], [], []
    ctx = hp.Context(min(chunk, count), n, n, device=dev.index)
    for c0 in range(0, count, chunk):
        B = min(chunk, count - c0)
        u, v, fl = W.training_case(B, n, seed0 + c0)
        ud = torch.from_numpy(u.astype(np.float32)).to(dev)
        vd = torch.from_numpy(v.astype(np.float32)).to(dev)
        fd = torch.from_numpy(fl).to(dev)
        div = hp.hp_divergence(ud, vd, fd)
        divs.append(div); fls.append(fd); tgts.append(hp.hp_jacobi_target(ctx, div, fd, sweeps))
    ctx.close()
    return torch.cat(divs), torch.cat(fls), torch.cat(tgts)


def train(cnn: hp.CNN, data, epochs: int = 20, batch: int = 64, lr: float = 1e-3,
          lambda_div: float = 0.1, seed: int = 0, log_every: int = 0):
    """Adam over shuffled mini-batches; returns the per-step losses."""
    div, fl, tgt = data
    N, ny, nx = div.shape
    trainer = hp.Trainer(cnn, batch, ny, nx)
    g = np.random.default_rng(seed)
    steps = (N // batch) * epochs
    losses = torch.empty(max(steps, 1), dtype=torch.float64, device=div.device)
    k_step = 0
    for ep in range(epochs):
        order = torch.from_numpy(g.permutation(N)).to(div.device)
        for k in range(0, N - batch + 1, batch):
            idx = order[k:k + batch]
            trainer.step(div[idx].contiguous(), fl[idx].contiguous(), tgt[idx].contiguous(),
                         lr=lr, lambda_div=lambda_div, loss_out=losses[k_step:k_step + 1])
            k_step += 1
            if log_every and k_step % log_every == 0:
                print(f"step {k_step} loss {losses[k_step - 1].item():.4e}", flush=True)
    trainer.sync_params()
    trainer.close()
    return losses[:k_step].cpu().numpy().tolist()


# Physics-driven training (Sec. 3.2, Eq. 4)
#
# Reading: the short-term term is the divergence left by the network at
# t + 1, the long-term term the one it leaves at t + n after the training
# solver (network-only projection, then advection) has run n - 1 steps from
# the same state; n = 4 nine times in ten, else 16.  Advection is not
# differentiated and the rolled-out state is an input of the long-term term,
# so both terms are one-step losses through the same network, on the state at
# t and on the state reached at t + n - 1.

def pdnn_rollout(cnn: hp.CNN, ctx: hp.Context, u, v, flags, steps: int, dt: float = 0.1,
                 trace: list | None = None):
    """The intermediate velocity u*_{t+steps} reached from u*_t = (u, v) by
    `steps` steps of the training solver: the network-only projection (guess
    s * CNN(div / s, flags), Eq. 2, no Jacobi sweep), then semi-Lagrangian
    self-advection without buoyancy (the training flows carry no density
    variation).  The inputs are not modified.  With a list as `trace`, every
    step appends (u*, v*, projected u, projected v) before advecting."""
    prm = hp.ProjectParams(threshold=0.0, max_iters=0, dt=dt)
    adv = hp.PlumeParams(dt=dt, gravity=0.0)
    rho = torch.ones(flags.shape, dtype=torch.float32, device=flags.device)
    cu, cv = u.clone(), v.clone()
    for _ in range(steps):
        before = (cu.clone(), cv.clone()) if trace is not None else None
        hp.hp_project_hybrid(ctx, cnn, cu, cv, flags, prm)
        if trace is not None:
            trace.append((*before, cu.clone(), cv.clone()))
        cu, cv, rho = hp.hp_advect_step(cu, cv, rho, flags, adv)
    return cu, cv


def pdnn_batch(cnn: hp.CNN, ctx: hp.Context, u, v, flags, n: int, alpha: float = 1.0,
               beta: float = 1.0, dt: float = 0.1):
    """(div, flags, weight) of one physics-driven step on B grids: the grids
    at t with weight alpha / B and the same grids rolled out to t + n - 1
    with weight beta / B (2B grids, for Trainer.pdnn_step)."""
    B = flags.shape[0]
    ul, vl = pdnn_rollout(cnn, ctx, u, v, flags, n - 1, dt)
    div = torch.cat([hp.hp_divergence(u, v, flags), hp.hp_divergence(ul, vl, flags)])
    w = torch.cat([torch.full((B,), alpha / B), torch.full((B,), beta / B)])
    return div, torch.cat([flags, flags]), w.to(device=flags.device, dtype=torch.float32)


def train_pdnn(cnn: hp.CNN, data, steps: int, batch: int = 32, lr: float = 1e-3,
               alpha: float = 1.0, beta: float = 1.0, norm: int = 1, dt: float = 0.1,
               p_long: float = 0.1, n_short: int = 4, n_long: int = 16, seed: int = 0):
    """Adam on the physics-driven loss over random mini-batches of velocity
    states (u, v, flags on the device, u and v with divergence); the network
    object must hold 2 * batch grids.  Returns the per-step losses and the
    rollout lengths drawn."""
    u, v, fl = data
    N, ny, nx = fl.shape
    ctx = hp.Context(batch, ny, nx, device=fl.device.index)
    trainer = hp.Trainer(cnn, 2 * batch, ny, nx)
    g = np.random.default_rng(seed)
    losses = torch.empty(max(steps, 1), dtype=torch.float64, device=fl.device)
    ns = []
    for k in range(steps):
        idx = torch.from_numpy(g.choice(N, batch, replace=False)).to(fl.device)
        n = n_long if g.random() < p_long else n_short
        ns.append(n)
        div, f2, w = pdnn_batch(cnn, ctx, u[idx].contiguous(), v[idx].contiguous(),
                                fl[idx].contiguous(), n, alpha, beta, dt)
        trainer.pdnn_step(div, f2, w, norm=norm, lr=lr, loss_out=losses[k:k + 1])
    trainer.sync_params()
    trainer.close()
    ctx.close()
    return losses[:steps].cpu().numpy().tolist(), ns
