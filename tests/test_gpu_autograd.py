"""Differentiation form: the energy as a torch.autograd.Function with a
hand-written backward, dE/dx = -F and dE/dq = phi, on the 20,001-charge water
box (L = 58.5 A, r_c = 9 A, 48^3 grid).

Checks:
  - the backward against the FP64 oracle's gradient (rms relative 1e-5, the
    FP32 path's force tolerance);
  - against central finite differences of the GPU energy on 200 random atoms
    and 200 random charges.  At h = 1e-4 (A, e) the difference of two FP32
    evaluations carries rounding noise: about 450 neighbours' FP32 potentials
    change between the two runs, 6e-8 relative each, so the energy difference is
    uncertain by ~3e-7 and the quotient by ~2e-3 absolute (forces here are
    O(1) e^2/A^2).  The h = 1e-4 check uses 1e-2 absolute + 1e-2 relative; at
    h = 1e-2 the noise falls 100-fold and the O(h^2) truncation is ~1e-4, so
    that check uses 1e-3 relative to the rms gradient.
"""
import numpy as np
import pytest

import oracle as O
from paper_1911_01377_gb300 import build as B
from paper_1911_01377_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    B.build()
    from paper_1911_01377_gb300.usr import USeries
    w = W.get("water_20k")
    ctx = USeries(w.box, w.grid, 9.0, "C1_B2", max_atoms=w.n)
    return torch, w, ctx


def _energy(torch, ctx, xyz, q):
    from paper_1911_01377_gb300.autograd import usr_energy
    return usr_energy(xyz, q, ctx)


def test_backward_matches_oracle_gradient(setup):
    torch, w, ctx = setup
    xyz = torch.from_numpy(w.xyzq[:, :3].copy()).cuda().requires_grad_(True)
    q = torch.from_numpy(w.xyzq[:, 3].copy()).cuda().requires_grad_(True)
    E = _energy(torch, ctx, xyz, q)
    E.backward()
    from tests.golden import paper_tables
    ref = O.evaluate(O.Series(*paper_tables()["table2_C1"]), 9.0, w.box, w.xyzq[:, :3], w.xyzq[:, 3])
    gx = xyz.grad.cpu().numpy().astype(np.float64)
    gq = q.grad.cpu().numpy().astype(np.float64)
    assert abs(E.item() / ref.E - 1.0) < 1e-6
    assert O.rms_rel(gx, -ref.F) < 1e-5
    assert O.rms_rel(gq, ref.phi) < 1e-5


def test_backward_scales_with_upstream_gradient(setup):
    torch, w, ctx = setup
    xyz = torch.from_numpy(w.xyzq[:, :3].copy()).cuda().requires_grad_(True)
    q = torch.from_numpy(w.xyzq[:, 3].copy()).cuda().requires_grad_(True)
    (3.0 * _energy(torch, ctx, xyz, q)).backward()
    g3 = xyz.grad.clone()
    xyz.grad = None
    _energy(torch, ctx, xyz, q).backward()
    assert torch.allclose(g3, 3.0 * xyz.grad, rtol=1e-6, atol=0)


@pytest.mark.parametrize("h,rtol,atol", [(1e-4, 1e-2, 1e-2), (1e-2, 1e-3, 0.0)])
def test_central_finite_differences(setup, h, rtol, atol):
    torch, w, ctx = setup
    rng = np.random.default_rng(1911)
    atoms = rng.choice(w.n, size=200, replace=False)
    base = torch.from_numpy(w.xyzq.copy()).cuda()
    xyz = base[:, :3].clone().requires_grad_(True)
    q = base[:, 3].clone().requires_grad_(True)
    _energy(torch, ctx, xyz, q).backward()
    gx = xyz.grad.cpu().numpy().astype(np.float64)
    gq = q.grad.cpu().numpy().astype(np.float64)
    scale_x = np.sqrt(np.mean(gx ** 2))
    scale_q = np.sqrt(np.mean(gq ** 2))

    def E_of(t):
        out, en = ctx.eval(t)
        return float(en[0].item())

    fd_x, an_x, fd_q, an_q = [], [], [], []
    for i in atoms:
        a = int(rng.integers(3))
        p = base.clone(); p[i, a] += h
        m = base.clone(); m[i, a] -= h
        # the perturbed coordinates as the GPU sees them (float32)
        hh = float(p[i, a].item()) - float(m[i, a].item())
        fd_x.append((E_of(p) - E_of(m)) / hh)
        an_x.append(gx[i, a])
        p = base.clone(); p[i, 3] += h
        m = base.clone(); m[i, 3] -= h
        hq = float(p[i, 3].item()) - float(m[i, 3].item())
        fd_q.append((E_of(p) - E_of(m)) / hq)
        an_q.append(gq[i])
    fd_x, an_x, fd_q, an_q = map(np.array, (fd_x, an_x, fd_q, an_q))
    assert np.all(np.abs(fd_x - an_x) <= atol * scale_x + rtol * np.maximum(np.abs(an_x), scale_x))
    assert np.all(np.abs(fd_q - an_q) <= atol * scale_q + rtol * np.maximum(np.abs(an_q), scale_q))
