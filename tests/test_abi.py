"""The C ABI without a GPU: the library builds and loads, exports every entry
point include/usr.h declares, and its host-side planning agrees with the
paper and the oracle (no kernel is launched here)."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import oracle as O
from oracle import series as S
from paper_1911_01377_gb300 import build as B
from paper_1911_01377_gb300 import usr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libusr():
    B.build()
    return usr.lib()


def _declared():
    text = open(os.path.join(ROOT, "include", "usr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(usr_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(libusr):
    names = _declared()
    assert "usr_eval" in names and "usr_init" in names
    for name in names:
        assert hasattr(libusr, name), name


def test_presets_are_the_paper_tables(libusr, tables):
    keys = ["table2_C0", "table2_C1", "table2_C2", "table1_a", "table1_b", "table1_c"]
    for pid, key in enumerate(keys):
        s = usr.usr_series_preset(pid)
        b, r0, w0, s0 = tables[key]
        assert (s.b, s.r0, s.w0, s.s0) == (b, r0, w0, s0)
        assert s.n_terms == 0 and s.trunc_eps == 0.0
    with pytest.raises(usr.UsrError):
        usr.usr_series_preset(6)


@pytest.mark.parametrize("r_c", [8.0, 9.0, 10.0, 13.0])
def test_plan_matches_closed_forms(libusr, tables, r_c):
    box, grid = (80.0, 80.0, 100.0), (64, 64, 80)
    info = usr.usr_plan(usr.make_params(box, grid, r_c, "C1_B2", max_atoms=10))
    ser = O.Series(*tables["table2_C1"])
    assert abs(info.sigma - r_c / ser.r0) < 1e-14 * info.sigma
    assert abs(info.F0 / O.F0(ser, r_c) - 1.0) < 1e-13
    # Eq. 33: smallest N with the bound below 1e-9
    N = next(N for N in range(1, 17) if S.trunc_bound(N, ser.b, r_c / ser.r0, max(box)) <= 1e-9)
    assert info.n_terms == N
    assert abs(info.trunc_bound / S.trunc_bound(N, ser.b, r_c / ser.r0, max(box)) - 1.0) < 1e-9
    assert list(info.cells) == [int(math.floor(L / r_c)) for L in box]
    assert list(info.h) == [L / n for L, n in zip(box, grid)]
    # the pair kernel's polynomial for the wide terms of F: within 5e-9 of F(0), below FP32 rounding
    assert info.poly_max_err < 5e-9


def test_plan_rejects_unsupported_input(libusr):
    ok = dict(box=(31.0, 31.0, 31.0), grid=(32, 32, 32), r_c=9.0, series="C1_B2")
    usr.usr_plan(usr.make_params(**ok))
    usr.usr_plan(usr.make_params(**dict(ok, conv=1)))
    usr.usr_plan(usr.make_params(**dict(ok, grid=(36, 32, 32), conv=1)))
    usr.usr_plan(usr.make_params(**dict(ok, conv=2)))
    bad = [dict(ok, r_c=11.0),                    # fewer than 3 cells on an axis
           dict(ok, r_c=-1.0),
           dict(ok, grid=(32, 16, 32)),           # fewer than spread_points + 8 points
           dict(ok, box=(31.0, 0.0, 31.0)),
           dict(ok, spread_sigma_over_h=3.5),     # sigma_0^2 <= 2 sigma_s^2
           dict(ok, grid=(30, 32, 32), conv=1),   # TF32x3 needs grid dims that are multiples of 4
           dict(ok, grid=(36, 32, 32), conv=2)]   # BF16x3 needs multiples of 8
    for kw in bad:
        with pytest.raises(usr.UsrError) as e:
            usr.usr_plan(usr.make_params(**kw))
        assert e.value.code == 2
    for kw in [dict(ok, spread_points=7), dict(ok, spread_points=18), dict(ok, conv=5),
               dict(ok, series=(0.9, 2.0, 1.0, 1.0))]:
        with pytest.raises(usr.UsrError) as e:
            usr.usr_plan(usr.make_params(**kw))
        assert e.value.code == 1
    assert usr.usr_status_string(0) == "ok"
    assert "capacity" in usr.usr_status_string(7)


def test_plan_limits(libusr):
    # the stated limits: at most 4096 grid points per axis and 2^31 - 1 in all and box sides of at most
    # 1e5 A (USR_ERR_BOX), 2^28 atoms
    # per context (USR_ERR_CAPACITY), a series whose full term table stays within 4096 terms (b >= 1.0113,
    # USR_ERR_ARG); a box-to-cutoff ratio beyond int range is refused, not converted
    ok = dict(box=(31.0, 31.0, 31.0), grid=(32, 32, 32), r_c=9.0, series="C1_B2")
    usr.usr_plan(usr.make_params(**dict(ok, max_atoms=1 << 28)))
    usr.usr_plan(usr.make_params(**dict(ok, series=(1.012, 2.0, 1.0, 1.0), n_terms=3)))
    usr.usr_plan(usr.make_params(**dict(ok, box=(9.9e4, 300.0, 300.0), grid=(4096, 32, 32), r_c=80.0,
                                        spread_points=8, spread_sigma_over_h=0.83)))
    cases = [(dict(ok, grid=(4100, 32, 32)), 2),
             (dict(ok, box=(4000.0, 4000.0, 4000.0), grid=(2048, 2048, 1024)), 2),
             (dict(ok, max_atoms=(1 << 28) + 1), 7),
             (dict(ok, series=(1.01, 2.0, 1.0, 1.0), n_terms=3), 1),
             (dict(ok, box=(1e300, 1e300, 1e300), r_c=1e-300), 2),
             (dict(ok, box=(1.2e5, 300.0, 300.0), grid=(4096, 32, 32), r_c=80.0, spread_points=8,
                   spread_sigma_over_h=0.83), 2)]
    for kw, code in cases:
        with pytest.raises(usr.UsrError) as e:
            usr.usr_plan(usr.make_params(**kw))
        assert e.value.code == code, kw


def test_init_without_gpu_fails_cleanly(libusr):
    # with no usable device the context cannot be created; the error is a
    # status code, not a crash (on a GPU machine this creates a context)
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(usr.UsrError) as e:
        usr.usr_init(usr.make_params((31.0,) * 3, (32,) * 3, 9.0, "C1_B2", max_atoms=100))
    assert e.value.code in (4, 5)


def test_null_context_arguments_are_refused(libusr):
    # entry points that read a context refuse a NULL one with USR_ERR_ARG before touching the device
    q = ctypes.c_double(7.0)
    assert libusr.usr_net_charge(None, ctypes.addressof(q), None) == 1
    assert q.value == 7.0
    assert libusr.usr_virial(None, ctypes.addressof(q), None) == 1
    assert libusr.usr_last_device_status(None) == 1


def test_binding_has_every_entry_point(libusr):
    # the Python binding carries every entry point of the C ABI under the same name
    missing = [name for name in _declared() if not callable(getattr(usr, name, None))]
    assert not missing, missing


def test_server_entry_points_without_a_server(libusr):
    # the serving entry points check their arguments before touching the device: a NULL server is refused,
    # and so are parameters out of range (these run without a GPU)
    import torch
    for kw in (dict(slots=65), dict(hbm_budget_bytes=-1.0)):
        with pytest.raises(usr.UsrError) as e:
            usr.usr_server_create(**kw)
        assert e.value.code == 1
    assert usr.usr_server_poll(0) == [] and usr.usr_server_poll(0, 0) == []
    for call in (lambda: usr.usr_server_wait(0, 0.1), lambda: usr.usr_server_info(0)):
        with pytest.raises(usr.UsrError) as e:
            call()
        assert e.value.code == 1
    usr.usr_server_destroy(0)                                  # NULL is ignored
    srv = usr.Server.__new__(usr.Server)
    srv.handle, srv._live = 0, {}
    p = usr.make_params((31.0,) * 3, (32,) * 3, 9.0, "C1_B2", max_atoms=10)
    x, o, e4 = torch.zeros((10, 4)), torch.zeros((10, 4)), torch.zeros(4, dtype=torch.float64)
    with pytest.raises(usr.UsrError) as e:
        srv.submit(p, x, o, e4)
    assert e.value.code == 1 and srv._live == {}
    assert srv.poll() == []


class _FakeServerLib:
    """Stands in for libusr's serving entry points: records submissions and completes them in order."""

    def __init__(self):
        self.pending, self.next = [], 0

    def usr_server_create(self, p, h):
        assert p._obj.slots == 3 and p._obj.hbm_budget_bytes == 1e9
        h._obj.value = 1234
        return 0

    def usr_server_submit(self, s, p, n, x, o, e, t):
        assert s == 1234 and n == 10 and x and o and e and p._obj.max_atoms == 10
        t._obj.value = self.next
        self.pending.append(self.next)
        self.next += 1
        return 0

    def usr_server_poll(self, s, tk, lat, st, m):
        k = min(m, len(self.pending))
        for i in range(k):
            tk[i], lat[i], st[i] = self.pending[i], 0.5 + i, 0
        self.pending = self.pending[k:]
        return k

    def usr_server_wait(self, s, t):
        return 0 if s == 1234 else 1

    def usr_server_info(self, s, b, q, f):
        b._obj.value, q._obj.value, f._obj.value = 7.0, 1, 2
        return 0

    def usr_server_destroy(self, s):
        assert s == 1234


def test_server_wrapper_bookkeeping(libusr, monkeypatch):
    # the Server class marshals through the usr_server_* wrappers and keeps each request's tensors referenced
    # until poll() returns its ticket (the library itself replaced by a fake: no GPU)
    import torch
    p = usr.make_params((31.0,) * 3, (32,) * 3, 9.0, "C1_B2", max_atoms=10)
    monkeypatch.setattr(usr, "_lib", _FakeServerLib())
    srv = usr.Server(hbm_budget_bytes=1e9, slots=3)
    x, o, e = torch.zeros((10, 4)), torch.zeros((10, 4)), torch.zeros(4, dtype=torch.float64)
    assert (srv.submit(p, x, o, e), srv.submit(p, x, o, e)) == (0, 1) and set(srv._live) == {0, 1}
    srv.wait(5)
    assert srv.info() == (7.0, 1, 2)
    assert srv.poll(1) == [(0, 0.5, 0)] and set(srv._live) == {1}
    assert srv.poll() == [(1, 0.5, 0)] and srv._live == {}
    srv.close()
    assert srv.handle == 0


def test_binding_refuses_unusable_tensors():
    # the binding checks every tensor whose pointer it hands to the library before any library call: wrong
    # side (host / device), dtype, layout or size raise ValueError (runs without a GPU: every case fails
    # before a context is touched)
    import torch
    ctx = usr.USeries.__new__(usr.USeries)
    ctx.ctx, ctx._last_n = 0, None
    x = torch.zeros((10, 4), dtype=torch.float32)
    bad_device = [x, torch.zeros((10, 4), dtype=torch.float64), x.t(), torch.zeros(40, dtype=torch.float32)]
    for t in bad_device:
        with pytest.raises(ValueError):
            ctx.eval(t)
        with pytest.raises(ValueError):
            ctx.debug_cells(t)
        with pytest.raises(ValueError):
            ctx.debug_pairs(t)
    for t in [x.double(), x.t(), x.reshape(40), x[:, :3].contiguous(), "not a tensor"]:
        with pytest.raises(ValueError):
            ctx.eval_host(t)
    with pytest.raises(ValueError):                                   # out too small
        ctx.eval_host(x, out=torch.zeros((9, 4), dtype=torch.float32))
    with pytest.raises(ValueError):                                   # energy too small / wrong dtype
        ctx.eval_host(x, out=torch.zeros((10, 4), dtype=torch.float32), energy=torch.zeros(3, dtype=torch.float64))
    with pytest.raises(ValueError):
        ctx.eval_host(x, out=torch.zeros((10, 4), dtype=torch.float32), energy=torch.zeros(4, dtype=torch.float32))
    with pytest.raises(ValueError):                                   # parts() only after an evaluation of n rows
        ctx.parts(10)
    srv = usr.Server.__new__(usr.Server)
    srv.handle, srv._live = 0, {}
    p = usr.make_params((31.0,) * 3, (32,) * 3, 9.0, "C1_B2", max_atoms=10)
    for args in [(x.double(), torch.zeros((10, 4))), (x, torch.zeros((10, 3))), (x, torch.zeros((10, 4)).double()),
                 (x, torch.zeros((10, 4)), torch.zeros(2, dtype=torch.float64))]:
        with pytest.raises(ValueError):
            srv.submit(p, *args)


def test_static_cell_list_refuses_oversized_cell_counts(libusr):
    """usr_cells_static checks every cell factor before multiplying, so a product that would overflow
    64 bits is refused as a capacity error before any device call (null buffers: nothing is touched)."""
    for cells in [(2_097_152, 2_097_152, 2_097_152), (65_537, 1, 1), (256, 256, 2), (1 << 30, 1 << 30, 4)]:
        with pytest.raises(usr.UsrError) as e:
            usr.usr_cells_static(4, None, (10.0, 10.0, 10.0), cells, None, None, None, None, 0)
        assert e.value.code == 7
    with pytest.raises(usr.UsrError) as e:          # mean occupancy above 2,048 atoms per cell
        usr.usr_cells_static(2049 * 27, None, (10.0, 10.0, 10.0), (3, 3, 3), None, None, None, None, 0)
    assert e.value.code == 7


def test_multilevel_plan(libusr):
    """The multilevel option moves the wide terms to the coarse grid (the threshold is on the deconvolved
    width: at least 2.25 coarse spacings on every axis); it needs even grid sizes and no virial."""
    box, grid = (220.0,) * 3, (176,) * 3
    plain = usr.usr_plan(usr.make_params(box, grid, 10.0, "C1_B2", max_atoms=10, conv=2))
    ml = usr.usr_plan(usr.make_params(box, grid, 10.0, "C1_B2", max_atoms=10, conv=2, multilevel=1))
    assert plain.n_terms_coarse == 0
    assert ml.n_terms == plain.n_terms and 0 < ml.n_terms_coarse < ml.n_terms
    assert ml.trunc_bound == plain.trunc_bound
    for kw in [dict(grid=(176, 176, 175)), dict(virial=1)]:
        args = dict(box=box, grid=grid, r_c=10.0, series="C1_B2", max_atoms=10, multilevel=1)
        args.update(kw)
        with pytest.raises(usr.UsrError) as e:
            usr.usr_plan(usr.make_params(**args))
        assert e.value.code == 2
    with pytest.raises(usr.UsrError) as e:
        usr.usr_plan(usr.make_params(box, grid, 10.0, "C1_B2", max_atoms=10, multilevel=2))
    assert e.value.code == 1


def test_autograd_refuses_unusable_inputs():
    # the differentiable energy checks its inputs before any evaluation (runs without a GPU)
    import torch
    from paper_1911_01377_gb300.autograd import usr_energy
    xyz, q = torch.zeros((5, 3)), torch.zeros(5)
    with pytest.raises(TypeError):
        usr_energy(xyz, q, None)                                  # host tensors
    with pytest.raises(TypeError):
        usr_energy(xyz.double(), q.double(), None)
