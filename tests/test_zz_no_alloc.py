"""usr_cells_static: the cell list built without any device allocation.

This entry point is for callers that cannot call cudaMalloc when they need a
cell list (an application that owns all GPU memory through a fixed pool, code
inside allocator callbacks or hand-built CUDA graphs, a tool injected into
another program).  Its temporaries live in one fixed device array inside the
library.  The test checks, through the C ABI, that two calls in a row give
exactly the cell list of the context-based entry point (usr_debug_cells): cell
lists are integer and index work, so the comparison is bit for bit.  The
second call is smaller than the first, so contents left in the shared array by
the first call must not leak into the second.

This file is named to be collected last: if it fails, a run that stops at the
first failure has already run every other test.
"""
import numpy as np
import pytest

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


def _static_cells(torch, xyzq, box, cells, stream=None):
    n = xyzq.shape[0]
    ncell = int(np.prod(cells))
    cell = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    perm = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    start = torch.full((ncell + 1,), -7, dtype=torch.int32, device="cuda")
    xw = torch.full((max(n, 1), 4), float("nan"), dtype=torch.float32, device="cuda")
    usr.usr_cells_static(n, xyzq.data_ptr(), box, cells, cell.data_ptr(), perm.data_ptr(), start.data_ptr(),
                         xw.data_ptr(), stream)
    return cell[:n], perm[:n], start, xw[:n]


def _same(torch, a, b):
    torch.cuda.synchronize()
    for x, y in zip(a, b):
        x, y = x.cpu().numpy(), y.cpu().numpy()
        assert x.shape == y.shape
        assert np.array_equal(x.view(np.int32), y.view(np.int32))


def test_static_cell_list_matches_context_entry_point(torch_cuda):
    torch = torch_cuda
    runs = [(W.get("membrane_slab"), 9.0), (W.get("water_3k"), 9.0)]   # large first, then smaller
    for w, r_c in runs:
        ctx = usr.USeries(w.box, w.grid, r_c, "C1_B2", max_atoms=w.n)
        cells = list(ctx.info.cells)
        x = torch.from_numpy(w.xyzq).cuda()
        ref = ctx.debug_cells(x)
        got = _static_cells(torch, x, w.box, cells)
        _same(torch, got, ref)
        ctx.close()


def test_static_cell_list_limits(torch_cuda):
    torch = torch_cuda
    x = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(usr.UsrError) as e:
        usr.usr_cells_static(262_145, x.data_ptr(), (10.0, 10.0, 10.0), (3, 3, 3), x.data_ptr(), x.data_ptr(),
                             x.data_ptr(), x.data_ptr())
    assert e.value.code == 7                     # USR_ERR_CAPACITY
    with pytest.raises(usr.UsrError) as e:
        usr.usr_cells_static(4, x.data_ptr(), (10.0, 10.0, 10.0), (64, 64, 17), x.data_ptr(), x.data_ptr(),
                             x.data_ptr(), x.data_ptr())
    assert e.value.code == 7


def test_static_cell_list_on_a_side_stream_and_empty(torch_cuda):
    """A call enqueued on a non-default stream gives the same list as the context entry point on that
    stream; n = 0 writes cell_start as all zeros."""
    torch = torch_cuda
    w = W.get("water_3k")
    ctx = usr.USeries(w.box, w.grid, 9.0, "C1_B2", max_atoms=w.n)
    cells = list(ctx.info.cells)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        x = torch.from_numpy(w.xyzq).cuda()
        ref = ctx.debug_cells(x, stream=s)
        got = _static_cells(torch, x, w.box, cells, stream=s.cuda_stream)
    s.synchronize()
    _same(torch, got, ref)
    ctx.close()
    empty = torch.zeros((1, 4), dtype=torch.float32, device="cuda")
    _, _, start, _ = _static_cells(torch, empty[:0], w.box, cells)
    torch.cuda.synchronize()
    assert np.array_equal(start.cpu().numpy(), np.zeros(int(np.prod(cells)) + 1, dtype=np.int32))
