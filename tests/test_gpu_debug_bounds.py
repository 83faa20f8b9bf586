"""The bounds-checking debug build (USR_DEBUG_BOUNDS): every kernel checks the
indices it computes against the sizes of the buffers it addresses and records a
violation in the status word instead of making the access.  One small system
(48 charges, ragged grid, tensor-core and FP32 convolutions, virial on) runs
through that build in a separate process: no index may be out of range, and the
results must still match the FP64 oracle.
"""
import os
import subprocess
import sys

import pytest

from paper_1911_01377_gb300 import build as B

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import numpy as np, torch
import oracle as O
from paper_1911_01377_gb300 import usr, workloads as W
from tests.golden import paper_tables
box = (19.3, 21.1, 23.7)
xyzq = W.random_neutral(11, 48, box, min_dist=1.2)
ref = O.evaluate(O.Series(*paper_tables()["table2_C1"]), 6.0, box, xyzq[:, :3], xyzq[:, 3])
for conv, grid in ((0, (30, 33, 37)), (2, (32, 32, 40))):
    ctx = usr.USeries(box, grid, 6.0, "C1_B2", max_atoms=64, conv=conv, virial=1)
    out, en = ctx.eval(torch.from_numpy(xyzq).cuda())
    cnt, _ = ctx.debug_pairs(torch.from_numpy(xyzq).cuda())
    torch.cuda.synchronize()
    st = usr.usr_last_device_status(ctx.ctx)
    assert st == 0, f"status {st} (conv {conv})"
    e = abs(float(en[0].item()) / ref.E - 1.0)
    f = O.rms_rel(out.cpu().numpy().astype(np.float64)[:, :3], ref.F)
    assert e < 1e-6 and f < 1e-5, (conv, e, f)
    ctx.close()
print("DEBUG_BOUNDS_OK")
"""


def test_small_system_under_bounds_checks():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    lib = B.build(debug_bounds=True)
    env = dict(os.environ, USR_LIBRARY=lib, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and "DEBUG_BOUNDS_OK" in r.stdout, r.stdout + r.stderr
