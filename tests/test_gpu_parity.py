"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.  Cell and pair lists are compared bit for bit; energies,
forces and potentials within the tolerances stated here:

  total (near + far + self), FP32 path vs same-parameter oracle:
      energy relative error <= 1e-6, rms relative force and potential error <= 1e-5
  near part alone (Eq. 20, FP32 pair arithmetic): rms relative <= 2e-6
  far part alone (grid spreading + per-axis convolutions + interpolation):
      potential <= 2e-5, force <= 1e-4 (rms relative to the far part itself)

"rms relative" is sqrt(sum |x - x_ref|^2 / sum |x_ref|^2).
"""
import functools
import math

import numpy as np
import pytest

import oracle as O
from paper_1911_01377_gb300 import build as B
from paper_1911_01377_gb300 import usr
from paper_1911_01377_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_E = 1e-6
TOL_F = 1e-5
TOL_PHI = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    B.build()
    return torch


def ragged_random():
    box = (27.3, 31.7, 36.1)
    xyzq = W.random_neutral(42, 1500, box, min_dist=1.2)
    return W.Workload("ragged_random_1500", box, (30, 35, 41), (8.5,), xyzq, "1500 random charges, ragged grid")


WORKLOADS = {
    "water_3k": lambda: W.get("water_3k"),
    "ragged": ragged_random,
    "water_20k": lambda: W.get("water_20k"),
}


@functools.lru_cache(maxsize=None)
def workload(name):
    return WORKLOADS[name]() if name in WORKLOADS else W.get(name)


@functools.lru_cache(maxsize=None)
def oracle_result(name, r_c, preset="table2_C1"):
    from tests.golden import paper_tables
    w = workload(name)
    ser = O.Series(*paper_tables()[preset])
    return O.evaluate(ser, r_c, w.box, w.xyzq[:, :3], w.xyzq[:, 3])


def gpu_eval(torch, w, r_c, series="C1_B2", keep_parts=True, **kw):
    ctx = usr.USeries(w.box, w.grid, r_c, series, max_atoms=max(w.n, 1), **kw)
    usr.usr_set_keep_parts(ctx.ctx, keep_parts)
    x = torch.from_numpy(w.xyzq).cuda()
    out, en = ctx.eval(x)
    near = far = None
    if keep_parts and w.n:
        near, far = ctx.parts(w.n)
    torch.cuda.synchronize()
    assert usr.usr_last_device_status(ctx.ctx) == 0
    res = dict(out=out.cpu().numpy().astype(np.float64), E=en.cpu().numpy(),
               near=None if near is None else near.cpu().numpy().astype(np.float64),
               far=None if far is None else far.cpu().numpy().astype(np.float64))
    return ctx, res


def _ncell(ctx):
    return ctx.info.cells[0] * ctx.info.cells[1] * ctx.info.cells[2]


@pytest.mark.parametrize("name,r_c", [("water_3k", 9.0), ("ragged", 8.5), ("membrane_slab", 8.0),
                                      ("membrane_slab", 13.0)])
def test_cell_list_bit_exact(torch_cuda, name, r_c):
    torch = torch_cuda
    w = workload(name)
    ctx = usr.USeries(w.box, w.grid, r_c, "C1_B2", max_atoms=w.n)
    cell, perm, start, xw = ctx.debug_cells(torch.from_numpy(w.xyzq).cuda())
    torch.cuda.synchronize()
    ocell, oxw = O.canon_cells(w.xyzq, w.box, list(ctx.info.cells))
    cell = cell.cpu().numpy()
    assert np.array_equal(cell, ocell)
    order = np.lexsort((np.arange(w.n), ocell))                  # by cell, then caller index
    assert np.array_equal(perm.cpu().numpy(), order)
    counts = np.bincount(ocell, minlength=_ncell(ctx))
    assert np.array_equal(start.cpu().numpy(), np.concatenate([[0], np.cumsum(counts)]))
    xw = xw.cpu().numpy()
    assert np.array_equal(xw[:, :3].view(np.int32), oxw[order].view(np.int32))
    assert np.array_equal(xw[:, 3], w.xyzq[order, 3])


@pytest.mark.parametrize("name,r_c", [("water_3k", 9.0), ("ragged", 8.5), ("membrane_slab", 10.0)])
def test_pair_list_bit_exact(torch_cuda, name, r_c):
    torch = torch_cuda
    w = workload(name)
    ctx = usr.USeries(w.box, w.grid, r_c, "C1_B2", max_atoms=w.n)
    cnt, h = ctx.debug_pairs(torch.from_numpy(w.xyzq).cuda())
    torch.cuda.synchronize()
    ocnt, oh = O.canon_pairs(w.xyzq, w.box, list(ctx.info.cells), r_c)
    assert np.array_equal(cnt.cpu().numpy(), ocnt)
    assert np.array_equal(h.cpu().numpy().view(np.uint64), oh)


@pytest.mark.parametrize("name,r_c", [("water_3k", 9.0), ("ragged", 8.5), ("water_20k", 9.0)])
def test_parts_parity(torch_cuda, name, r_c):
    w = workload(name)
    ref = oracle_result(name, r_c)
    _, g = gpu_eval(torch_cuda, w, r_c)
    assert O.rms_rel(g["near"][:, 3], ref.phi_near) < 2e-6
    assert O.rms_rel(g["near"][:, :3], ref.F_near) < 2e-6
    assert O.rms_rel(g["far"][:, 3], ref.phi_far) < 2e-5
    assert O.rms_rel(g["far"][:, :3], ref.F_far) < 1e-4
    # part energies relative to the magnitude of their terms, 1/2 sum |q_i phi_i|
    # (a part's sum can cancel to far below its terms, e.g. E_near of random charges)
    q = w.xyzq[:, 3].astype(np.float64)
    scale_near = 0.5 * np.sum(np.abs(q * ref.phi_near))
    scale_far = 0.5 * np.sum(np.abs(q * ref.phi_far))
    assert abs(g["E"][1] - ref.E_near) < 2e-6 * scale_near
    assert abs(g["E"][2] - ref.E_far) < 2e-5 * scale_far
    assert abs(g["E"][3] / ref.E_self - 1.0) < 1e-6


@pytest.mark.parametrize("name,r_c", [("water_3k", 9.0), ("ragged", 8.5), ("water_20k", 9.0)])
def test_total_parity(torch_cuda, name, r_c):
    w = workload(name)
    ref = oracle_result(name, r_c)
    ctx, g = gpu_eval(torch_cuda, w, r_c)
    assert abs(g["E"][0] / ref.E - 1.0) < TOL_E
    assert O.rms_rel(g["out"][:, :3], ref.F) < TOL_F
    assert O.rms_rel(g["out"][:, 3], ref.phi) < TOL_PHI
    assert abs(g["E"][0] - (g["E"][1] + g["E"][2] + g["E"][3])) < 1e-12 * abs(g["E"][0])
    # neutral inputs (up to the FP32 rounding of the charges): the net charge diagnostic is their exact sum
    q = w.xyzq[:, 3].astype(np.float64)
    assert abs(ctx.net_charge() - q.sum()) < 1e-9 * np.abs(q).sum()


@pytest.mark.parametrize("r_c", [8.0, 13.0])
def test_membrane_slab_full_size(torch_cuda, r_c):
    # the benchmark's workload and launch configuration, full oracle
    w = workload("membrane_slab")
    ref = oracle_result("membrane_slab", r_c)
    _, g = gpu_eval(torch_cuda, w, r_c, keep_parts=False)
    assert abs(g["E"][0] / ref.E - 1.0) < TOL_E
    assert O.rms_rel(g["out"][:, :3], ref.F) < TOL_F
    assert O.rms_rel(g["out"][:, 3], ref.phi) < TOL_PHI


@pytest.mark.parametrize("r_c", [8.0, 13.0])
def test_benchmark_timed_form_full_size(torch_cuda, r_c):
    # the form bench.py times, at its launch configuration: BF16x3 tensor-core convolutions, the GSE-style
    # spreading of Sec. IV.A (8-point stencil, sigma_s = 0.83 h), full slab; the metric's bound is an rms
    # relative force error <= 1e-4 against the same-parameter oracle, energy within 1e-6
    w = workload("membrane_slab")
    ref = oracle_result("membrane_slab", r_c)
    _, g = gpu_eval(torch_cuda, w, r_c, keep_parts=False, conv=2, spread_points=8, spread_sigma_over_h=0.83)
    assert abs(g["E"][0] / ref.E - 1.0) < 1e-6
    assert O.rms_rel(g["out"][:, :3], ref.F) < 1e-4
    assert O.rms_rel(g["out"][:, 3], ref.phi) < 1e-4


def test_wrapping_and_images(torch_cuda):
    # shifting atoms by whole box vectors changes nothing beyond rounding
    torch = torch_cuda
    w = workload("water_3k")
    ref = oracle_result("water_3k", 9.0)
    rng = np.random.default_rng(3)
    shifted = w.xyzq.copy()
    k = rng.integers(-3, 4, size=(w.n, 3)).astype(np.float32)
    shifted[:, :3] = (shifted[:, :3].astype(np.float64) + k * np.array(w.box)).astype(np.float32)
    ws = W.Workload("shifted", w.box, w.grid, w.r_c, shifted)
    _, g = gpu_eval(torch, ws, 9.0)
    assert abs(g["E"][0] / ref.E - 1.0) < 5 * TOL_E
    assert O.rms_rel(g["out"][:, :3], ref.F) < 5 * TOL_F


def test_boundary_coordinates(torch_cuda):
    # atoms exactly on and just inside the box faces, and at negative zero
    torch = torch_cuda
    L = 24.0
    box = (L, L, L)
    pts = [(0.0, 0.0, 0.0, 0.5), (L, 3.0, 4.0, -0.5), (np.nextafter(np.float32(L), np.float32(0)), 5.0, 6.0, 0.25),
           (-0.0, 7.0, 8.0, -0.25), (-1e-7, 11.0, 12.0, 0.3), (12.0, -L, 2 * L, -0.3)]
    base = W.random_neutral(9, 400, box, min_dist=1.5)
    xyzq = np.concatenate([base, np.array(pts, dtype=np.float32)], axis=0).astype(np.float32)
    w = W.Workload("faces", box, (28, 28, 28), (7.5,), xyzq)
    ctx = usr.USeries(box, w.grid, 7.5, "C1_B2", max_atoms=w.n)
    cell, perm, start, xw = ctx.debug_cells(torch.from_numpy(xyzq).cuda())
    ocell, oxw = O.canon_cells(xyzq, box, list(ctx.info.cells))
    assert np.array_equal(cell.cpu().numpy(), ocell)
    ref = O.evaluate(O.Series(*usr_series_tuple("C1_B2")), 7.5, box, xyzq[:, :3], xyzq[:, 3])
    _, g = gpu_eval(torch, w, 7.5)
    assert abs(g["E"][0] / ref.E - 1.0) < TOL_E
    assert O.rms_rel(g["out"][:, :3], ref.F) < TOL_F


def usr_series_tuple(name):
    from tests.golden import paper_tables
    key = {"C0_B2": "table2_C0", "C1_B2": "table2_C1", "C2_B2": "table2_C2"}[name]
    return paper_tables()[key]


def test_dense_cells_and_non_neutral(torch_cuda):
    # > 128 atoms in some cells (multi-chunk staging) and a net charge
    torch = torch_cuda
    box = (30.0, 30.0, 30.0)
    rng = np.random.default_rng(17)
    cluster = rng.random((700, 3)) * 8.0 + 1.0
    rest = rng.random((800, 3)) * 30.0
    pos = np.concatenate([cluster, rest])
    q = rng.normal(0.0, 0.2, size=pos.shape[0]) + 0.01
    xyzq = np.concatenate([pos, q[:, None]], axis=1).astype(np.float32)
    w = W.Workload("dense", box, (32, 32, 32), (9.0,), xyzq)
    ref = O.evaluate(O.Series(*usr_series_tuple("C1_B2")), 9.0, box, xyzq[:, :3], xyzq[:, 3])
    ctx, g = gpu_eval(torch, w, 9.0)
    assert abs(g["E"][0] / ref.E - 1.0) < 1e-5
    assert O.rms_rel(g["out"][:, :3], ref.F) < TOL_F
    assert O.rms_rel(g["out"][:, 3], ref.phi) < 1e-5
    # the net charge diagnostic: sum q of the FP32 charges (about 15 e here); one charge more or less
    # (|q| ~ 0.2) is far outside the tolerance
    qf = xyzq[:, 3].astype(np.float64)
    assert abs(ctx.net_charge() - qf.sum()) < 1e-9 * np.abs(qf).sum()


@pytest.mark.parametrize("preset", ["C0_B2", "C2_B2"])
def test_other_constructions(torch_cuda, preset):
    w = workload("water_3k")
    ref = O.evaluate(O.Series(*usr_series_tuple(preset)), 9.0, w.box, w.xyzq[:, :3], w.xyzq[:, 3])
    _, g = gpu_eval(torch_cuda, w, 9.0, series=preset)
    assert abs(g["E"][0] / ref.E - 1.0) < TOL_E
    assert O.rms_rel(g["out"][:, :3], ref.F) < TOL_F


# tensor-core convolution forms (USR_CONV_TF32X3 = 1, USR_CONV_BF16X3 = 2).  TF32x3
# keeps about 21 mantissa bits per operand, so it is held to the FP32 path's
# tolerances; BF16x3 keeps about 16 bits (relative 2^-17 per operand), about
# 1e-5 per convolution pass, and is held to the benchmark's force bound 1e-4.
TC_TOL = {1: dict(E=1e-6, F=1e-5, phi=1e-5), 2: dict(E=2e-5, F=1e-4, phi=1e-4)}


@pytest.mark.parametrize("conv", [1, 2])
@pytest.mark.parametrize("name,r_c", [("water_3k", 9.0), ("water_20k", 9.0), ("membrane_slab", 10.0)])
def test_tensor_core_convolution_parity(torch_cuda, conv, name, r_c):
    w = workload(name)
    ref = oracle_result(name, r_c)
    _, g = gpu_eval(torch_cuda, w, r_c, conv=conv)
    tol = TC_TOL[conv]
    assert abs(g["E"][0] / ref.E - 1.0) < tol["E"]
    assert O.rms_rel(g["out"][:, :3], ref.F) < tol["F"]
    assert O.rms_rel(g["out"][:, 3], ref.phi) < tol["phi"]
    # the near part does not depend on the convolution form
    assert O.rms_rel(g["near"][:, 3], ref.phi_near) < 2e-6


@pytest.mark.parametrize("conv", [1, 2])
def test_tensor_core_ragged_lines(torch_cuda, conv):
    # line counts that are not multiples of the 128-line tile, more than one N
    # tile on an axis (n + 1 > 256 needs two), and a non-cubic box
    torch = torch_cuda
    box = (22.4, 27.2, 288.0)
    xyzq = W.random_neutral(77, 2400, box, min_dist=1.3)
    w = W.Workload("tc_ragged", box, (24, 32, 264), (7.0,), xyzq, "tensor-core ragged shapes")
    ref = O.evaluate(O.Series(*usr_series_tuple("C1_B2")), 7.0, w.box, w.xyzq[:, :3], w.xyzq[:, 3])
    _, gtc = gpu_eval(torch, w, 7.0, conv=conv)
    tol = TC_TOL[conv]
    assert O.rms_rel(gtc["far"][:, 3], ref.phi_far) < 2 * tol["F"]
    assert O.rms_rel(gtc["out"][:, :3], ref.F) < tol["F"]
    # the z pass here contracts K = 7 terms x 264 points = 1848 per output on the
    # tensor cores, whose FP32 accumulation rounds differently from the FP32
    # path's; the energy of these 2,400 random unit-variance charges is a small
    # residual (E_far = 1.85 E), so the check is relative to the far energy
    assert abs(gtc["E"][0] - ref.E) < 2 * tol["F"] * abs(ref.E_far)


def test_tiny_and_empty(torch_cuda):
    torch = torch_cuda
    box = (25.0, 25.0, 25.0)
    ctx = usr.USeries(box, (24, 24, 24), 8.0, "C1_B2", max_atoms=4)
    x = torch.zeros((0, 4), dtype=torch.float32, device="cuda")
    out = torch.zeros((1, 4), dtype=torch.float32, device="cuda")
    en = torch.full((4,), 7.0, dtype=torch.float64, device="cuda")
    usr.usr_eval(ctx.ctx, 0, x.data_ptr(), out.data_ptr(), en.data_ptr())
    torch.cuda.synchronize()
    assert en.cpu().tolist() == [0.0, 0.0, 0.0, 0.0]
    assert ctx.net_charge() == 0.0
    # a single charge: self term plus its periodic far images, k = 0 dropped
    one = np.array([[3.0, 4.0, 5.0, 0.7]], dtype=np.float32)
    ref = O.evaluate(O.Series(*usr_series_tuple("C1_B2")), 8.0, box, one[:, :3], one[:, 3])
    o, e = ctx.eval(torch.from_numpy(one).cuda())
    torch.cuda.synchronize()
    assert abs(e[0].item() / ref.E - 1.0) < 1e-5
    assert abs(o[0, 3].item() / ref.phi[0] - 1.0) < 1e-5
    assert ctx.net_charge() == float(np.float32(0.7))
    # capacity is enforced
    big = torch.zeros((5, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(usr.UsrError) as err:
        ctx.eval(big)
    assert err.value.code == 7


def test_nonfinite_sets_status(torch_cuda):
    torch = torch_cuda
    w = workload("water_3k")
    x = w.xyzq.copy()
    x[5, 1] = np.nan
    ctx = usr.USeries(w.box, w.grid, 9.0, "C1_B2", max_atoms=w.n)
    ctx.eval(torch.from_numpy(x).cuda())
    assert usr.usr_last_device_status(ctx.ctx) == 3
    assert usr.usr_last_device_status(ctx.ctx) == 0          # cleared
    ctx.eval(torch.from_numpy(w.xyzq).cuda())
    assert usr.usr_last_device_status(ctx.ctx) == 0


def test_positions_beyond_the_wrap_are_refused(torch_cuda):
    """Far outside the box (1e10 A and more here, over 1e8 box lengths) the single-precision wrap's period
    count floorf(x * (1/L)) is off by several periods, so one correction cannot bring the wrapped value into
    [0, L].  Such a row is refused like a non-finite one: the status reads USR_ERR_NONFINITE and the row is
    evaluated as a zero charge at the origin, bit for bit as if it had been given that way; the next
    evaluation on the context is clean.  One far row per evaluation: refused rows all go to the origin, and
    two charges at one point (r = 0) are themselves reported as non-finite by the pair kernel."""
    torch = torch_cuda
    w = workload("water_3k")
    ctx = usr.USeries(w.box, w.grid, 9.0, "C1_B2", max_atoms=w.n)
    for row, ax, x in ((5, 0, 1e10), (6, 1, -1e30), (7, 2, 3.3e13)):
        far = w.xyzq.copy()
        far[row, ax] = x
        L = w.box[ax]
        k = np.floor(far[row, ax] * np.float32(1.0 / L))     # the wrap's period count, in FP32
        assert abs(float(k) - float(far[row, ax]) / L) > 3.0
        origin = w.xyzq.copy()
        origin[row] = 0.0
        o_far, e_far = ctx.eval(torch.from_numpy(far).cuda())
        o_far, e_far = o_far.cpu().numpy(), e_far.cpu().numpy()
        assert usr.usr_last_device_status(ctx.ctx) == 3
        assert usr.usr_last_device_status(ctx.ctx) == 0      # cleared
        o_org, e_org = ctx.eval(torch.from_numpy(origin).cuda())
        o_org, e_org = o_org.cpu().numpy(), e_org.cpu().numpy()
        assert usr.usr_last_device_status(ctx.ctx) == 0
        assert np.array_equal(o_far.view(np.int32), o_org.view(np.int32))
        assert np.array_equal(e_far.view(np.int64), e_org.view(np.int64))


def test_eval_host_matches_device(torch_cuda):
    # the host-buffer entry point runs the same kernels: identical bits
    torch = torch_cuda
    w = workload("water_3k")
    ctx = usr.USeries(w.box, w.grid, 9.0, "C1_B2", max_atoms=w.n)
    od, ed = ctx.eval(torch.from_numpy(w.xyzq).cuda())
    xh = torch.from_numpy(w.xyzq).pin_memory()
    oh, eh = ctx.eval_host(xh)
    torch.cuda.synchronize()
    assert np.array_equal(oh.numpy(), od.cpu().numpy())
    assert np.array_equal(eh.numpy(), ed.cpu().numpy())


@pytest.mark.parametrize("name,r_c", [("water_3k", 9.0), ("ragged", 8.5), ("membrane_slab", 11.0)])
def test_repeatable(torch_cuda, name, r_c):
    # no atomics decide a floating-point order anywhere on the path: two
    # evaluations of the same input agree bit for bit
    torch = torch_cuda
    w = workload(name)
    ctx = usr.USeries(w.box, w.grid, r_c, "C1_B2", max_atoms=w.n)
    x = torch.from_numpy(w.xyzq).cuda()
    o1, e1 = ctx.eval(x)
    o1 = o1.clone(); e1 = e1.clone()
    o2, e2 = ctx.eval(x)
    torch.cuda.synchronize()
    assert np.array_equal(o1.cpu().numpy(), o2.cpu().numpy())
    assert np.array_equal(e1.cpu().numpy(), e2.cpu().numpy())


@pytest.mark.parametrize("conv", [0, 2])
def test_streams_and_concurrent_contexts(torch_cuda, conv):
    # the evaluation forks its far part onto the context's own stream and joins it back: on a caller stream that
    # is not the default one, and with two contexts evaluating at once on two streams, every result is the same,
    # bit for bit, as one evaluation alone on the default stream
    torch = torch_cuda
    w = workload("water_20k")
    x = torch.from_numpy(w.xyzq).cuda()
    ref_ctx = usr.USeries(w.box, w.grid, 9.0, "C1_B2", max_atoms=w.n, conv=conv)
    o_ref, e_ref = ref_ctx.eval(x)
    torch.cuda.synchronize()
    o_ref, e_ref = o_ref.cpu().numpy(), e_ref.cpu().numpy()
    ctxs = [usr.USeries(w.box, w.grid, 9.0, "C1_B2", max_atoms=w.n, conv=conv) for _ in range(2)]
    streams = [torch.cuda.Stream() for _ in range(2)]
    outs = []
    for _ in range(3):
        for c, s in zip(ctxs, streams):
            with torch.cuda.stream(s):
                outs.append(c.eval(x, stream=s.cuda_stream))
    torch.cuda.synchronize()
    for o, e in outs:
        assert np.array_equal(o.cpu().numpy(), o_ref)
        assert np.array_equal(e.cpu().numpy(), e_ref)
    for c in ctxs + [ref_ctx]:
        c.close()


@pytest.mark.parametrize("conv", [0, 2])
def test_cuda_graph_capture_and_replay(torch_cuda, conv):
    # usr_eval enqueues kernels and copies only (no allocation, no host
    # synchronisation), so it can be captured in a CUDA graph and replayed;
    # replays pick up new positions written into the same input buffer
    torch = torch_cuda
    w = workload("water_3k")
    ctx = usr.USeries(w.box, w.grid, 9.0, "C1_B2", max_atoms=w.n, conv=conv)
    x = torch.from_numpy(w.xyzq).cuda()
    out = torch.empty((w.n, 4), dtype=torch.float32, device="cuda")
    en = torch.empty(4, dtype=torch.float64, device="cuda")
    ctx.eval(x, out, en)
    torch.cuda.synchronize()
    ref_o, ref_e = out.clone(), en.clone()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            usr.usr_eval(ctx.ctx, w.n, x.data_ptr(), out.data_ptr(), en.data_ptr(), torch.cuda.current_stream())
    torch.cuda.synchronize()
    out.zero_()
    en.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, ref_o) and torch.equal(en, ref_e)
    moved = w.xyzq.copy()
    moved[:, :3] += np.float32(0.37)
    x.copy_(torch.from_numpy(moved))
    g.replay()
    torch.cuda.synchronize()
    o2, e2 = ctx.eval(torch.from_numpy(moved).cuda())
    torch.cuda.synchronize()
    assert torch.equal(out, o2) and torch.equal(en, e2)
