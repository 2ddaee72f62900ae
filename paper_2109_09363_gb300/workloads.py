"""Seeded synthetic inputs for the projection workloads.

This module only draws input fields (velocities, densities, obstacle flags)
with numpy's PCG64; it holds none of the method's arithmetic (no divergence,
no Laplacian, no correction).  The same arrays feed the CUDA path and the FP64
oracle, so no random-number parity between the two is needed.

Grid conventions: u has shape [B][ny][nx+1] (face (j, i) sits at x = i,
y = j + 1/2), v has shape [B][ny+1][nx] (face (j, i) at x = i + 1/2, y = j),
cell (i, j) is centred at (i + 1/2, j + 1/2), row 0 is the top of the image and
flags != 0 marks a solid cell.
"""
from __future__ import annotations

import numpy as np


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def vortex_velocity(ny: int, nx: int, seed: int, n_vortices: int = 32, amp=(-1.0, 1.0),
                    width=(4.0, 32.0)):
    """Sum of Gaussian vortices sampled point-wise on the faces (FP64).

    Each vortex has a centre uniform in the domain, amplitude A ~ U(amp) and
    width sigma ~ U(width); its velocity is (-A (y-cy)/sigma, A (x-cx)/sigma)
    * exp(-r^2 / 2 sigma^2).
    """
    g = _rng(seed)
    cx = g.uniform(0, nx, n_vortices)
    cy = g.uniform(0, ny, n_vortices)
    a = g.uniform(amp[0], amp[1], n_vortices)
    s = g.uniform(width[0], width[1], n_vortices)
    xu, yu = np.meshgrid(np.arange(nx + 1, dtype=np.float64), np.arange(ny) + 0.5)
    xv, yv = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny + 1, dtype=np.float64))
    u = np.zeros((ny, nx + 1))
    v = np.zeros((ny + 1, nx))
    for k in range(n_vortices):
        ru = ((xu - cx[k]) ** 2 + (yu - cy[k]) ** 2) / (2 * s[k] ** 2)
        rv = ((xv - cx[k]) ** 2 + (yv - cy[k]) ** 2) / (2 * s[k] ** 2)
        u += -a[k] * (yu - cy[k]) / s[k] * np.exp(-ru)
        v += a[k] * (xv - cx[k]) / s[k] * np.exp(-rv)
    return u, v


def random_obstacles(ny: int, nx: int, seed: int, n_range=(1, 6), rect_side=(16, 96),
                     disc_radius=(8, 48), count=None):
    """uint8 flags with 1-6 solid rectangles or discs (50/50), centres uniform."""
    g = _rng(seed)
    n = int(g.integers(n_range[0], n_range[1] + 1)) if count is None else int(count)
    x, y = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny) + 0.5)
    fl = np.zeros((ny, nx), np.uint8)
    for _ in range(n):
        cx, cy = g.uniform(0, nx), g.uniform(0, ny)
        if g.uniform() < 0.5:
            w, h = g.uniform(rect_side[0], rect_side[1], 2)
            fl[(np.abs(x - cx) <= w / 2) & (np.abs(y - cy) <= h / 2)] = 1
        else:
            r = g.uniform(disc_radius[0], disc_radius[1])
            fl[(x - cx) ** 2 + (y - cy) ** 2 <= r * r] = 1
    return fl


def batched_vortex_case(batch: int, n: int, seed0: int = 0, n_vortices: int = 32):
    """B independent n x n grids: vortex velocity + random obstacles, seeds seed0..seed0+B-1.

    Returns (u [B][n][n+1], v [B][n+1][n], flags [B][n][n]) as FP64 / uint8.
    """
    us, vs, fs = [], [], []
    for b in range(batch):
        u, v = vortex_velocity(n, n, 1000 + seed0 + b, n_vortices=n_vortices)
        fl = random_obstacles(n, n, 2000 + seed0 + b)
        us.append(u); vs.append(v); fs.append(fl)
    return np.stack(us), np.stack(vs), np.stack(fs)


def plume_flags(n: int, cylinder_radius: float = 0.0, cylinder_height: float = 0.0):
    """Closed box, optional solid disc centred cylinder_height cells above the inlet row."""
    fl = np.zeros((n, n), np.uint8)
    if cylinder_radius > 0:
        x, y = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5)
        cx, cy = n / 2.0, (n - 0.5) - cylinder_height
        fl[(x - cx) ** 2 + (y - cy) ** 2 <= cylinder_radius ** 2] = 1
    return fl


def inlet_columns(n: int, width: int | None = None):
    """[start, stop) columns of the density inlet strip centred in the bottom row."""
    w = n // 8 if width is None else width
    return n // 2 - w // 2, n // 2 - w // 2 + w


def paper_plume_geometry(n: int, cylinder: bool = True):
    """The plume cases of Sec. 2.1 on an n x n box: an inlet centred in the
    bottom face whose width is 0.29 n (the paper's D_in, which its R = 74.25
    at n = 512 makes a diameter), and optionally a solid disc of diameter
    0.312 n centred horizontally, its centre 0.625 n above the bottom wall.
    Returns (flags [n][n], (x0, x1) inlet columns)."""
    fl = plume_flags(n, cylinder_radius=0.156 * n if cylinder else 0.0,
                     cylinder_height=0.625 * n - 0.5)
    return fl, inlet_columns(n, width=int(round(0.29 * n)))


def plume_initial_state(n: int, seed: int = 0, noise_std: float = 1e-4):
    """rho = 1 + N(0, noise_std^2) per cell, u = v = 0 (FP64)."""
    g = _rng(seed)
    rho = 1.0 + noise_std * g.standard_normal((n, n))
    return np.zeros((n, n + 1)), np.zeros((n + 1, n)), rho


def source_velocity(ny: int, nx: int, seed: int, n_sources: int = 8, amp=(-1.0, 1.0),
                    width=(2.0, 12.0)):
    """Irrotational part with divergence: the face-sampled gradient of a sum of
    Gaussian potential bumps, psi = sum A exp(-r^2 / 2 sigma^2) (FP64)."""
    g = _rng(seed)
    cx = g.uniform(0, nx, n_sources)
    cy = g.uniform(0, ny, n_sources)
    a = g.uniform(amp[0], amp[1], n_sources)
    s = g.uniform(width[0], width[1], n_sources)
    xu, yu = np.meshgrid(np.arange(nx + 1, dtype=np.float64), np.arange(ny) + 0.5)
    xv, yv = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny + 1, dtype=np.float64))
    u = np.zeros((ny, nx + 1))
    v = np.zeros((ny + 1, nx))
    for k in range(n_sources):
        eu = np.exp(-((xu - cx[k]) ** 2 + (yu - cy[k]) ** 2) / (2 * s[k] ** 2))
        ev = np.exp(-((xv - cx[k]) ** 2 + (yv - cy[k]) ** 2) / (2 * s[k] ** 2))
        u += -a[k] * (xu - cx[k]) / s[k] ** 2 * eu
        v += -a[k] * (yv - cy[k]) / s[k] ** 2 * ev
    return u, v


def training_case(batch: int, n: int, seed0: int = 0):
    """Training inputs: vortex velocity plus Gaussian divergence sources, 0-4
    obstacles (rectangles / discs sized to the grid); seeds seed0.. per grid.
    Returns (u [B][n][n+1], v [B][n+1][n], flags [B][n][n]) FP64 / uint8."""
    us, vs, fs = [], [], []
    for b in range(batch):
        sd = seed0 + b
        u1, v1 = vortex_velocity(n, n, 5000 + sd, n_vortices=max(4, n // 8),
                                 width=(n / 32, n / 8))
        u2, v2 = source_velocity(n, n, 6000 + sd, n_sources=max(2, n // 16),
                                 width=(n / 32, n / 8))
        fl = random_obstacles(n, n, 8000 + sd, n_range=(0, 4), rect_side=(n / 16, n / 4),
                              disc_radius=(n / 32, n / 8))
        us.append(u1 + u2); vs.append(v1 + v2); fs.append(fl)
    return np.stack(us), np.stack(vs), np.stack(fs)


def random_cylinders(n: int, count: int, seed: int, radius=(32.0, 128.0), inlet=None,
                     clearance: float = 8.0, tries: int = 10000):
    """uint8 flags with `count` solid discs of radius U(radius), centres drawn
    until the discs overlap neither each other nor the walls nor the inlet
    (a band of the inlet's columns, `clearance` cells beyond each side, over
    the bottom rows up to the disc), all with `clearance` cells to spare."""
    g = _rng(seed)
    x, y = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5)
    fl = np.zeros((n, n), np.uint8)
    discs = []
    for _ in range(tries):
        if len(discs) == count:
            break
        r = g.uniform(radius[0], radius[1])
        cx, cy = g.uniform(r + clearance, n - r - clearance, 2)
        if any((cx - a) ** 2 + (cy - b) ** 2 < (r + c + clearance) ** 2 for a, b, c in discs):
            continue
        if inlet is not None and inlet[0] - clearance - r < cx < inlet[1] + clearance + r and \
                cy + r + clearance > n - 4 * clearance:
            continue
        discs.append((cx, cy, r))
    if len(discs) < count:
        raise ValueError(f"only {len(discs)} of {count} discs fit")
    for cx, cy, r in discs:
        fl[(x - cx) ** 2 + (y - cy) ** 2 <= r * r] = 1
    return fl
