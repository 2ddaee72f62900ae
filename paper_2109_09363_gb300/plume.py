"""Plume driver: inlet + advection + buoyancy (hp_advect_step), then the
pressure projection (hp_project), on B grids of ny x nx.  Thin orchestration
of the C ABI; every step runs in the library's kernels."""
from __future__ import annotations

from dataclasses import dataclass, field

import paper_2109_09363_gb300 as hp


@dataclass
class PlumeConfig:
    ny: int = 128
    nx: int = 128
    batch: int = 1
    dt: float = 0.1
    gravity: float = -0.002
    rho_amb: float = 1.0
    rho_in: float = 1.1
    inlet: tuple = (56, 72)
    threshold: float = 1e-3
    max_iters: int = 2000
    scheme: int = 0  # advection: 0 first-order semi-Lagrangian, 1 MacCormack
    project: dict = field(default_factory=dict)


class Plume:
    """State (u, v, rho) on the device and one step = advect, then project."""

    def __init__(self, cfg: PlumeConfig, u, v, rho, flags, phi0_fn=None, cnn=None):
        """phi0_fn(u, v, flags) gives the Jacobi guess; with a network (cnn)
        the projection is the hybrid one (guess from the network)."""
        self.cfg = cfg
        self.u, self.v, self.rho, self.flags = u, v, rho, flags
        self.ctx = hp.Context(cfg.batch, cfg.ny, cfg.nx, device=u.device.index)
        self.pp = hp.PlumeParams(cfg.dt, cfg.gravity, cfg.rho_amb, cfg.rho_in, cfg.inlet[0],
                                 cfg.inlet[1], cfg.scheme)
        self.prm = hp.ProjectParams(threshold=cfg.threshold, max_iters=cfg.max_iters,
                                    dt=cfg.dt, **cfg.project)
        self.phi0_fn = phi0_fn
        self.cnn = cnn
        self.out = None

    def advect(self):
        self.u, self.v, self.rho = hp.hp_advect_step(self.u, self.v, self.rho, self.flags, self.pp)

    def project(self):
        if self.cnn is not None:
            self.out = hp.hp_project_hybrid(self.ctx, self.cnn, self.u, self.v, self.flags,
                                            self.prm)
            return self.out
        phi0 = self.phi0_fn(self.u, self.v, self.flags) if self.phi0_fn else None
        self.out = hp.hp_project(self.ctx, self.u, self.v, self.flags, self.prm, phi0=phi0,
                                 out=None)
        return self.out

    def head(self, contrast: float | None = None):
        """Plume head (Sec. 4.1) per grid, normalised by the box size:
        (h_y, left extent, right extent) as float tensors [B]; the plume is
        every cell whose density contrast reaches `contrast` (default a tenth
        of the inlet's).  h_y = 0 and extents <= 0 when there is none."""
        c = 0.1 * abs(self.cfg.rho_in - self.cfg.rho_amb) if contrast is None else contrast
        o = hp.hp_plume_head(self.rho, self.cfg.rho_amb, c).double()
        ny, nx = self.cfg.ny, self.cfg.nx
        return ((ny - o[:, 0]) / ny, (nx / 2 - o[:, 1]) / nx, (o[:, 2] + 1 - nx / 2) / nx)

    def step(self):
        self.advect()
        return self.project()
