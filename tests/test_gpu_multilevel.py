"""Multilevel far part (usr_params.multilevel = 1): the wide Gaussian terms on a
grid twice as coarse, reached by Gaussian restriction and prolongation (Sec. V's
remark on multilevel summation for wider terms).  Checked against the FP64
oracle with the tolerances of the single-grid forms, and against the
single-grid evaluation of the same system: the two differ only by the
transfers' error (about 1e-7 of the wide terms, a few 1e-10 per axis in a 1D
check), so their far parts agree far inside the parity tolerances.
"""
import functools

import numpy as np
import pytest

import oracle as O
from paper_1911_01377_gb300 import build as B
from paper_1911_01377_gb300 import usr
from paper_1911_01377_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    B.build()
    return torch


def serving_sized():
    # one system of the serving stream's shape (about 100k charges at 0.1 per A^3, grid of about 1 A)
    for box, grid, r_c, xyzq in W.serving_stream(7, 1, n_min=100000, n_max=100000):
        return W.Workload("serving_100k", box, grid, (r_c,), xyzq, "serving-sized water box")


WORKLOADS = {"water_20k": lambda: W.get("water_20k"), "membrane_slab": lambda: W.get("membrane_slab"),
             "serving_100k": serving_sized}


@functools.lru_cache(maxsize=None)
def workload(name):
    return WORKLOADS[name]()


@functools.lru_cache(maxsize=None)
def oracle_result(name, r_c):
    from tests.golden import paper_tables
    w = workload(name)
    return O.evaluate(O.Series(*paper_tables()["table2_C1"]), r_c, w.box, w.xyzq[:, :3], w.xyzq[:, 3])


def run(torch, w, r_c, **kw):
    ctx = usr.USeries(w.box, w.grid, r_c, "C1_B2", max_atoms=w.n, **kw)
    usr.usr_set_keep_parts(ctx.ctx, True)
    out, en = ctx.eval(torch.from_numpy(w.xyzq).cuda())
    near, far = ctx.parts(w.n)
    torch.cuda.synchronize()
    assert usr.usr_last_device_status(ctx.ctx) == 0
    info = ctx.info
    res = dict(out=out.cpu().numpy().astype(np.float64), E=en.cpu().numpy(),
               far=far.cpu().numpy().astype(np.float64), n_coarse=info.n_terms_coarse, n_terms=info.n_terms)
    ctx.close()
    return res


# (workload, r_c, convolution form, spreading points, spreading width / h); the serving-sized box (grid
# spacing 1.04 A, r_c = 9 A) takes the 10-point stencil: at 8 points the spreading error alone is about
# 1.2e-4 of the far potential there, with or without the coarse grid
CASES = [("water_20k", 9.0, 0, 0, 0.0), ("membrane_slab", 10.0, 0, 0, 0.0), ("membrane_slab", 10.0, 2, 8, 0.83),
         ("serving_100k", 9.0, 2, 10, 0.9), ("serving_100k", 9.0, 1, 10, 0.9)]


@pytest.mark.parametrize("name,r_c,conv,P,ratio", CASES)
def test_multilevel_against_oracle(torch_cuda, name, r_c, conv, P, ratio):
    w = workload(name)
    ref = oracle_result(name, r_c)
    kw = dict(conv=conv, spread_points=P, spread_sigma_over_h=ratio) if conv else dict(conv=conv)
    g = run(torch_cuda, w, r_c, multilevel=1, **kw)
    assert 0 < g["n_coarse"] < g["n_terms"]
    # the single-grid forms' bounds: FP32 1e-5 force / 1e-6 energy; BF16x3 with GSE spreading 1e-4 / 1e-6
    tol_f, tol_far_phi, tol_far_f = (1e-5, 2e-5, 1e-4) if conv == 0 else (1e-4, 1e-4, 1e-3)
    e = dict(E=abs(g["E"][0] / ref.E - 1.0), F=O.rms_rel(g["out"][:, :3], ref.F),
             far_phi=O.rms_rel(g["far"][:, 3], ref.phi_far), far_F=O.rms_rel(g["far"][:, :3], ref.F_far))
    print(f"\n{name} conv={conv} multilevel ({g['n_coarse']} of {g['n_terms']} terms coarse): "
          + " ".join(f"{k}={v:.2e}" for k, v in e.items()))
    assert e["E"] < 1e-6
    assert e["F"] < tol_f
    assert e["far_phi"] < tol_far_phi
    assert e["far_F"] < tol_far_f


@pytest.mark.parametrize("name,r_c", [("water_20k", 9.0), ("membrane_slab", 13.0)])
def test_multilevel_matches_single_grid(torch_cuda, name, r_c):
    w = workload(name)
    a = run(torch_cuda, w, r_c, multilevel=0)
    b = run(torch_cuda, w, r_c, multilevel=1)
    assert a["n_coarse"] == 0 and b["n_coarse"] > 0
    assert O.rms_rel(b["far"][:, 3], a["far"][:, 3]) < 2e-6
    assert O.rms_rel(b["far"][:, :3], a["far"][:, :3]) < 2e-5
    assert abs(b["E"][2] - a["E"][2]) < 2e-6 * abs(a["E"][2])
