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


def init_params(seed: int = 0) -> np.ndarray:
    """Initial parameters in the network's flat order (per layer weights
    [cout][cin][3][3] He-uniform, then zero biases), FP32."""
    g = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for cin, cout in LAYERS:
        lim = np.sqrt(6.0 / (9 * cin))
        parts.append(g.uniform(-lim, lim, 9 * cin * cout))
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
    prm = hp.ProjectParams(fixed_iters=sweeps)
    for c0 in range(0, count, chunk):
        B = min(chunk, count - c0)
        u, v, fl = W.training_case(B, n, seed0 + c0)
        ud = torch.from_numpy(u.astype(np.float32)).to(dev)
        vd = torch.from_numpy(v.astype(np.float32)).to(dev)
        fd = torch.from_numpy(fl).to(dev)
        div = hp.hp_divergence(ud, vd, fd)
        out = hp.hp_project(ctx, ud, vd, fd, prm)
        phi = out["p"].clone()
        nxt = hp.hp_jacobi_sweeps(ctx, phi, div, fd, 1)
        divs.append(div); fls.append(fd); tgts.append(0.5 * (phi + nxt))
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
