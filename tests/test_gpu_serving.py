"""Serving form: continuous batching of independent systems (usr_server_*).

Checks that every result is the same alone and in the mix: each system of a
mixed stream, evaluated by the server while other systems run on the device,
is compared with the same system evaluated alone by a fresh context.  The
evaluation path has no floating-point atomics, so the tolerance is exact
equality of every output bit.  Also: admission by the device-memory budget
(a budget that fits one system at a time still completes every request and
never holds more than the budget), a request that can never fit fails with
USR_ERR_OOM without stopping the others, and the result of one system is
checked against the FP64 oracle.
"""
import numpy as np
import pytest

import oracle as O
from paper_1911_01377_gb300 import build as B
from paper_1911_01377_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    B.build()
    from paper_1911_01377_gb300 import usr
    systems = list(W.serving_stream(2024, 12, n_min=2000, n_max=30000))
    return torch, usr, systems


FORMS = {"fp32": dict(conv=0), "serving": W.SERVING_FORM}


def _form(conv):
    return FORMS[conv] if isinstance(conv, str) else dict(conv=conv)


def _alone(torch, usr, box, grid, r_c, xyzq, conv, parts=False):
    ctx = usr.USeries(box, grid, r_c, "C1_B2", max_atoms=xyzq.shape[0], **_form(conv))
    if parts:
        usr.usr_set_keep_parts(ctx.ctx, True)
    out, en = ctx.eval(torch.from_numpy(xyzq).cuda())
    far = ctx.parts(xyzq.shape[0])[1] if parts else None
    torch.cuda.synchronize()
    assert usr.usr_last_device_status(ctx.ctx) == 0
    r = out.cpu().numpy(), en.cpu().numpy()
    if parts:
        r = r + (far.cpu().numpy(),)
    ctx.close()
    return r


def _serve(torch, usr, systems, conv, budget=0.0, slots=4):
    srv = usr.Server(hbm_budget_bytes=budget, slots=slots)
    bufs = []
    for box, grid, r_c, xyzq in systems:
        p = usr.make_params(box, grid, r_c, "C1_B2", max_atoms=xyzq.shape[0], **_form(conv))
        x = torch.from_numpy(xyzq).pin_memory()
        o = torch.empty((xyzq.shape[0], 4), dtype=torch.float32).pin_memory()
        e = torch.empty(4, dtype=torch.float64).pin_memory()
        t = srv.submit(p, x, o, e)
        bufs.append((t, o, e))
    srv.wait(timeout_s=120)
    done = {t: (lat, st) for t, lat, st in srv.poll()}
    held, queued, inflight = srv.info()
    srv.close()
    return bufs, done, held


@pytest.mark.parametrize("conv", [0, 2, "serving"])
def test_same_alone_and_in_the_mix(env, conv):
    torch, usr, systems = env
    bufs, done, _ = _serve(torch, usr, systems, conv)
    assert len(done) == len(systems)
    for (t, o, e), (box, grid, r_c, xyzq) in zip(bufs, systems):
        lat, st = done[t]
        assert st == 0 and lat > 0.0
        out, en = _alone(torch, usr, box, grid, r_c, xyzq, conv)
        assert np.array_equal(o.numpy(), out)
        assert np.array_equal(e.numpy(), en)


def test_budget_admission_and_oversized_request(env):
    torch, usr, systems = env
    sizes = []
    for box, grid, r_c, xyzq in systems:
        p = usr.make_params(box, grid, r_c, "C1_B2", max_atoms=xyzq.shape[0])
        sizes.append(usr.usr_plan(p).device_bytes)
    budget = 1.05 * max(sizes)                       # one system at a time at most
    big = W.serving_stream(99, 1, n_min=60000, n_max=60001)
    stream = systems[:5] + list(big)                 # the last one can never fit
    bufs, done, held = _serve(torch, usr, stream, 0, budget=budget, slots=4)
    assert held <= budget
    sts = [done[t][1] for t, _, _ in bufs]
    assert sts[:5] == [0] * 5
    assert sts[5] == 5                               # USR_ERR_OOM
    for (t, o, e), (box, grid, r_c, xyzq) in zip(bufs[:5], systems[:5]):
        out, en = _alone(torch, usr, box, grid, r_c, xyzq, 0)
        assert np.array_equal(o.numpy(), out)


def test_served_result_matches_oracle(env):
    torch, usr, systems = env
    box, grid, r_c, xyzq = min(systems, key=lambda s: s[3].shape[0])
    bufs, done, _ = _serve(torch, usr, [(box, grid, r_c, xyzq)], 0)
    (t, o, e), = bufs
    from tests.golden import paper_tables
    ref = O.evaluate(O.Series(*paper_tables()["table2_C1"]), r_c, box, xyzq[:, :3], xyzq[:, 3])
    assert abs(e.numpy()[0] / ref.E - 1.0) < 1e-6
    assert O.rms_rel(o.numpy()[:, :3].astype(np.float64), ref.F) < 1e-5


def test_serving_form_against_oracle(env):
    """The serving stream's form on a system of its largest sizes (100k charges, 96^3 grid of 1.04 A,
    r_c = 9 A), against the FP64 oracle with the bounds of the tensor-core forms (far potential 1e-4,
    far force 1e-3, total force 1e-4, energy 1e-6), and the same system through the server bit for bit."""
    torch, usr, _ = env
    (box, grid, r_c, xyzq), = W.serving_stream(7, 1, n_min=100000, n_max=100000)
    out, en, far = _alone(torch, usr, box, grid, r_c, xyzq, "serving", parts=True)
    from tests.golden import paper_tables
    ref = O.evaluate(O.Series(*paper_tables()["table2_C1"]), r_c, box, xyzq[:, :3], xyzq[:, 3])
    far = far.astype(np.float64)
    assert O.rms_rel(far[:, 3], ref.phi_far) < 1e-4
    assert O.rms_rel(far[:, :3], ref.F_far) < 1e-3
    assert O.rms_rel(out[:, :3].astype(np.float64), ref.F) < 1e-4
    assert abs(en[0] / ref.E - 1.0) < 1e-6
    bufs, done, _ = _serve(torch, usr, [(box, grid, r_c, xyzq)], "serving")
    (t, o, e), = bufs
    assert done[t][1] == 0
    assert np.array_equal(o.numpy(), out) and np.array_equal(e.numpy(), en)
