"""Virial tensor on the GPU against the FP64 oracle's (which is itself pinned by
Poisson summation and strain finite differences in test_oracle_energy.py).

W = -dE/d(strain) = W_near (pair sum, FP32 pair arithmetic) + W_far (six extra
grid convolution sets with derivative kernels, FP32).  Tolerance: the far part
carries the grid method's error, like E_far (which the FP32 path gets to a few
1e-7 relative); the check is 1e-5 of the largest component.
"""
import numpy as np
import pytest

import oracle as O
from paper_1911_01377_gb300 import build as B
from paper_1911_01377_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    B.build()
    return torch


def _ref(w, r_c):
    from tests.golden import paper_tables
    ser = O.Series(*paper_tables()["table2_C1"])
    wn, wf = O.virial(ser, r_c, w.box, w.xyzq[:, :3], w.xyzq[:, 3])
    return wn + wf


@pytest.mark.parametrize("name,r_c,conv", [("water_3k", 9.0, 0), ("water_3k", 9.0, 2), ("water_20k", 9.0, 0)])
def test_virial_matches_oracle(torch_cuda, name, r_c, conv):
    torch = torch_cuda
    from paper_1911_01377_gb300 import usr
    w = W.get(name)
    ctx = usr.USeries(w.box, w.grid, r_c, "C1_B2", max_atoms=w.n, conv=conv, virial=1)
    out, en = ctx.eval(torch.from_numpy(w.xyzq).cuda())
    Wg = ctx.virial().cpu().numpy()
    torch.cuda.synchronize()
    assert usr.usr_last_device_status(ctx.ctx) == 0
    ref = _ref(w, r_c)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(Wg - ref)) < 1e-5 * scale, (Wg, ref)
    assert np.array_equal(Wg, Wg.T)
    # the virial does not change the energy or forces of the evaluation
    ctx2 = usr.USeries(w.box, w.grid, r_c, "C1_B2", max_atoms=w.n, conv=conv)
    out2, en2 = ctx2.eval(torch.from_numpy(w.xyzq).cuda())
    torch.cuda.synchronize()
    assert torch.equal(out, out2) and torch.equal(en, en2)


def test_virial_ragged_box(torch_cuda):
    torch = torch_cuda
    from paper_1911_01377_gb300 import usr
    box = (27.3, 31.7, 36.1)
    xyzq = W.random_neutral(42, 1500, box, min_dist=1.2)
    w = W.Workload("ragged_random_1500", box, (30, 35, 41), (8.5,), xyzq, "ragged")
    ctx = usr.USeries(w.box, w.grid, 8.5, "C1_B2", max_atoms=w.n, virial=1)
    ctx.eval(torch.from_numpy(w.xyzq).cuda())
    Wg = ctx.virial().cpu().numpy()
    torch.cuda.synchronize()
    ref = _ref(w, 8.5)
    assert np.max(np.abs(Wg - ref)) < 1e-5 * np.max(np.abs(ref)), (Wg, ref)
