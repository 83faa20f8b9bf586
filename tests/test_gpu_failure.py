"""Failure path of the bounded device waits, exercised without any GPU fault.

Every wait of the tensor-core convolution kernel is bounded in time; when one
runs out, each CTA raises the timeout bit of the status word, waits for its
copies in flight, frees its tensor memory and returns.  usr_debug_inject_timeout
makes the next evaluation's first pass wait (1 ms) on a barrier that nothing
completes, so that path runs for real.  The test checks that the status reads
USR_ERR_TIMEOUT, that the context stays usable, and that the next evaluation is
bit-identical to one made before the injection and matches the FP64 oracle.
"""
import numpy as np
import pytest

import oracle as O
from paper_1911_01377_gb300 import build as B
from paper_1911_01377_gb300 import usr
from paper_1911_01377_gb300 import workloads as W

pytestmark = pytest.mark.gpu

USR_ERR_ARG = 1
USR_ERR_TIMEOUT = 6


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    B.build()
    return torch


@pytest.mark.parametrize("conv", [1, 2])
def test_wait_that_runs_out_reports_timeout_and_recovers(torch_cuda, conv):
    torch = torch_cuda
    w = W.get("water_3k")
    r_c = 9.0
    ctx = usr.USeries(w.box, w.grid, r_c, "C1_B2", max_atoms=w.n, conv=conv)
    x = torch.from_numpy(w.xyzq).cuda()
    out1, en1 = ctx.eval(x)
    torch.cuda.synchronize()
    assert usr.usr_last_device_status(ctx.ctx) == 0
    ref_o, ref_e = out1.clone(), en1.clone()

    usr.usr_debug_inject_timeout(ctx.ctx, True)
    ctx.eval(x)
    torch.cuda.synchronize()
    assert usr.usr_last_device_status(ctx.ctx) == USR_ERR_TIMEOUT

    out2, en2 = ctx.eval(x)
    torch.cuda.synchronize()
    assert usr.usr_last_device_status(ctx.ctx) == 0
    assert torch.equal(out2, ref_o) and torch.equal(en2, ref_e)
    from tests.golden import paper_tables
    ref = O.evaluate(O.Series(*paper_tables()["table2_C1"]), r_c, w.box, w.xyzq[:, :3], w.xyzq[:, 3])
    assert abs(float(en2[0].item()) / ref.E - 1.0) < 1e-6
    assert O.rms_rel(out2.cpu().numpy().astype(np.float64)[:, :3], ref.F) < 1e-5
    ctx.close()


def test_inject_needs_a_tensor_core_context(torch_cuda):
    w = W.get("water_3k")
    ctx = usr.USeries(w.box, w.grid, 9.0, "C1_B2", max_atoms=w.n, conv=0)
    with pytest.raises(usr.UsrError) as e:
        usr.usr_debug_inject_timeout(ctx.ctx, True)
    assert e.value.code == USR_ERR_ARG
    ctx.close()
