"""GPU adjoint of the fixed-count projection (hp_project_adjoint, through the
torch.autograd wrapper) against the FP64 adjoint oracle, which is itself pinned
by central differences and the dense Jacobian transpose.  Bar: 1e-5 of the
largest gradient entry (FP32 sweeps)."""
import numpy as np
import pytest

import oracle
from oracle import adjoint as AD
from paper_2109_09363_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
hp = pytest.importorskip("paper_2109_09363_gb300")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_09363_gb300 import build
    build.build()
    oracle.build()
    return torch.device("cuda:0")


@pytest.mark.parametrize("B,n,k", [(2, 64, 20), (1, 37, 0), (3, 50, 7)])
def test_adjoint_matches_oracle(dev, B, n, k):
    from paper_2109_09363_gb300.autograd import project_fixed
    dt, rho0 = 0.1, 1.0
    rng = np.random.default_rng(n + k)
    us, vs, fs = [], [], []
    for b in range(B):
        u, v = W.vortex_velocity(n, n, 60 + b, n_vortices=6, width=(2, n / 6))
        us.append(u); vs.append(v)
        fs.append(W.random_obstacles(n, n, 70 + b, rect_side=(3, n / 5), disc_radius=(2, n / 10)))
    u = np.stack(us).astype(np.float32); v = np.stack(vs).astype(np.float32); fl = np.stack(fs)
    phi0 = rng.standard_normal((B, n, n)).astype(np.float32)
    a = rng.standard_normal(u.shape).astype(np.float32)
    bb = rng.standard_normal(v.shape).astype(np.float32)
    c = rng.standard_normal(phi0.shape).astype(np.float32)
    ctx = hp.Context(B, n, n)
    ud = torch.from_numpy(u).to(dev).requires_grad_()
    vd = torch.from_numpy(v).to(dev).requires_grad_()
    pd = torch.from_numpy(phi0).to(dev).requires_grad_()
    fd = torch.from_numpy(fl).to(dev)
    uo, vo, po = project_fixed(ud, vd, pd, fd, ctx, k, dt, rho0)
    L = (uo * torch.from_numpy(a).to(dev)).sum() + (vo * torch.from_numpy(bb).to(dev)).sum() + \
        (po * torch.from_numpy(c).to(dev)).sum()
    L.backward()
    gus, gvs, gphi = AD.project_fixed_adjoint(a.astype(np.float64), bb.astype(np.float64),
                                              c.astype(np.float64), fl, k, dt, rho0)
    for got, exp in [(ud.grad, gus), (vd.grad, gvs), (pd.grad, gphi)]:
        g = got.cpu().numpy()
        assert np.abs(g - exp).max() <= 1e-5 * max(np.abs(exp).max(), 1e-30)
    # forward values agree with the oracle's fixed-count projection too
    ou, ov, op = AD.project_fixed(u.astype(np.float64), v.astype(np.float64),
                                  phi0.astype(np.float64), fl, k, dt, rho0)
    assert np.abs(uo.detach().cpu().numpy() - ou).max() <= 1e-5 * np.abs(ou).max()
