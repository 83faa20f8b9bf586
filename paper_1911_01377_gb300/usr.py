"""Python binding of libusr (include/usr.h): argument marshalling only.

Every function here has the name of the C entry point it calls; tensors are
passed as raw device pointers on the current PyTorch CUDA stream.  There is no
fallback: if libusr.so is missing or fails to load, `lib()` raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Tuple

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libusr.so")

_c_d = ctypes.c_double
_c_i = ctypes.c_int
_c_p = ctypes.c_void_p

USR_OK = 0
USR_NSTAGES = 7
# usr_conv: convolution form of the far part
USR_CONV_FP32, USR_CONV_TF32X3, USR_CONV_BF16X3 = 0, 1, 2
STAGES = ("bin", "near", "spread", "conv_x", "conv_y", "conv_z", "gather")
PRESETS = {"C0_B2": 0, "C1_B2": 1, "C2_B2": 2, "T1_A": 3, "T1_B": 4, "T1_C": 5}


class usr_series(ctypes.Structure):
    _fields_ = [("b", _c_d), ("r0", _c_d), ("w0", _c_d), ("s0", _c_d), ("n_terms", _c_i), ("trunc_eps", _c_d)]


class usr_params(ctypes.Structure):
    _fields_ = [("box", _c_d * 3), ("grid", _c_i * 3), ("r_c", _c_d), ("series", usr_series),
                ("spread_sigma_over_h", _c_d), ("spread_points", _c_i), ("conv", _c_i), ("max_atoms", _c_i),
                ("virial", _c_i), ("multilevel", _c_i)]


class usr_plan_info(ctypes.Structure):
    _fields_ = [("sigma", _c_d), ("F0", _c_d), ("spread_sigma", _c_d), ("h", _c_d * 3), ("trunc_bound", _c_d),
                ("n_terms", _c_i), ("cells", _c_i * 3), ("poly_degree", _c_i), ("n_explicit", _c_i),
                ("poly_max_err", _c_d), ("device_bytes", _c_d), ("n_terms_coarse", _c_i)]


class usr_server_params(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", _c_d), ("slots", _c_i)]


class UsrError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {usr_status_string(code)} (status {code})")


_lib = None


def lib():
    """Load libusr.so (built in-tree by paper_1911_01377_gb300.build)."""
    global _lib
    if _lib is None:
        # USR_LIBRARY names another build of the same library (the bounds-checking debug build)
        path = os.environ.get("USR_LIBRARY") or LIB_PATH
        if not os.path.exists(path):
            raise RuntimeError(f"libusr not found at {path}: run paper_1911_01377_gb300.build.build()")
        L = ctypes.CDLL(path)
        L.usr_series_preset.argtypes = [_c_i, ctypes.POINTER(usr_series)]
        L.usr_plan.argtypes = [ctypes.POINTER(usr_params), ctypes.POINTER(usr_plan_info)]
        L.usr_init.argtypes = [ctypes.POINTER(usr_params), ctypes.POINTER(_c_p)]
        L.usr_reconfigure.argtypes = [_c_p, ctypes.POINTER(usr_params), _c_p]
        L.usr_destroy.argtypes = [_c_p]
        L.usr_destroy.restype = None
        L.usr_info.argtypes = [_c_p, ctypes.POINTER(usr_plan_info)]
        L.usr_eval.argtypes = [_c_p, _c_i, _c_p, _c_p, _c_p, _c_p]
        L.usr_eval_host.argtypes = [_c_p, _c_i, _c_p, _c_p, _c_p, _c_p]
        L.usr_last_device_status.argtypes = [_c_p]
        L.usr_status_string.argtypes = [_c_i]
        L.usr_status_string.restype = ctypes.c_char_p
        L.usr_debug_cells.argtypes = [_c_p, _c_i, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p]
        L.usr_debug_pairs.argtypes = [_c_p, _c_i, _c_p, _c_p, _c_p, _c_p]
        L.usr_cells_static.argtypes = [_c_i, _c_p, ctypes.POINTER(_c_d), ctypes.POINTER(_c_i), _c_p, _c_p, _c_p,
                                       _c_p, _c_p]
        L.usr_eval_host_async.argtypes = [_c_p, _c_i, _c_p, _c_p, _c_p, _c_p]
        L.usr_server_create.argtypes = [ctypes.POINTER(usr_server_params), ctypes.POINTER(_c_p)]
        L.usr_server_submit.argtypes = [_c_p, ctypes.POINTER(usr_params), _c_i, _c_p, _c_p, _c_p,
                                        ctypes.POINTER(ctypes.c_longlong)]
        L.usr_server_poll.argtypes = [_c_p, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_c_d),
                                      ctypes.POINTER(_c_i), _c_i]
        L.usr_server_poll.restype = _c_i
        L.usr_server_wait.argtypes = [_c_p, _c_d]
        L.usr_server_info.argtypes = [_c_p, ctypes.POINTER(_c_d), ctypes.POINTER(ctypes.c_longlong),
                                      ctypes.POINTER(ctypes.c_longlong)]
        L.usr_server_destroy.argtypes = [_c_p]
        L.usr_server_destroy.restype = None
        L.usr_virial.argtypes = [_c_p, _c_p, _c_p]
        L.usr_net_charge.argtypes = [_c_p, _c_p, _c_p]
        L.usr_set_keep_parts.argtypes = [_c_p, _c_i]
        L.usr_debug_parts.argtypes = [_c_p, _c_p, _c_p, _c_p]
        L.usr_set_profiling.argtypes = [_c_p, _c_i]
        L.usr_stage_times.argtypes = [_c_p, ctypes.POINTER(ctypes.c_float)]
        L.usr_fp32_peak.argtypes = [ctypes.POINTER(_c_d)]
        L.usr_debug_inject_timeout.argtypes = [_c_p, _c_i]
        for name in ("usr_series_preset", "usr_plan", "usr_init", "usr_reconfigure", "usr_info", "usr_eval",
                     "usr_eval_host", "usr_eval_host_async", "usr_last_device_status", "usr_debug_cells",
                     "usr_debug_pairs", "usr_cells_static", "usr_set_keep_parts", "usr_virial", "usr_net_charge",
                     "usr_server_create", "usr_server_submit", "usr_server_wait", "usr_server_info", "usr_debug_parts",
                     "usr_set_profiling", "usr_stage_times", "usr_fp32_peak", "usr_debug_inject_timeout"):
            getattr(L, name).restype = _c_i
        _lib = L
    return _lib


def _check(code: int, where: str):
    if code != USR_OK:
        raise UsrError(code, where)


def usr_status_string(code: int) -> str:
    return lib().usr_status_string(code).decode()


def usr_series_preset(preset) -> usr_series:
    if isinstance(preset, str):
        preset = PRESETS[preset]
    s = usr_series()
    _check(lib().usr_series_preset(int(preset), ctypes.byref(s)), "usr_series_preset")
    return s


def make_params(box, grid, r_c, series, spread_sigma_over_h=0.0, spread_points=0, conv=0, max_atoms=0,
                n_terms=0, trunc_eps=0.0, virial=0, multilevel=0) -> usr_params:
    if isinstance(series, (str, int)):
        series = usr_series_preset(series)
    elif not isinstance(series, usr_series):
        b, r0, w0, s0 = tuple(series)[:4]
        series = usr_series(b, r0, w0, s0, 0, 0.0)
    series = usr_series(series.b, series.r0, series.w0, series.s0, int(n_terms or series.n_terms),
                        float(trunc_eps or series.trunc_eps))
    p = usr_params()
    p.box = (_c_d * 3)(*[float(v) for v in box])
    p.grid = (_c_i * 3)(*[int(v) for v in grid])
    p.r_c = float(r_c)
    p.series = series
    p.spread_sigma_over_h = float(spread_sigma_over_h)
    p.spread_points = int(spread_points)
    p.conv = int(conv)
    p.max_atoms = int(max_atoms)
    p.virial = int(virial)
    p.multilevel = int(multilevel)
    return p


def usr_plan(params: usr_params) -> usr_plan_info:
    info = usr_plan_info()
    _check(lib().usr_plan(ctypes.byref(params), ctypes.byref(info)), "usr_plan")
    return info


def usr_init(params: usr_params) -> int:
    h = _c_p()
    _check(lib().usr_init(ctypes.byref(params), ctypes.byref(h)), "usr_init")
    return h.value


def usr_reconfigure(ctx: int, params: usr_params, stream=None):
    _check(lib().usr_reconfigure(ctx, ctypes.byref(params), _stream_ptr(stream)), "usr_reconfigure")


def usr_destroy(ctx: int):
    lib().usr_destroy(ctx)


def usr_info(ctx: int) -> usr_plan_info:
    info = usr_plan_info()
    _check(lib().usr_info(ctx, ctypes.byref(info)), "usr_info")
    return info


def _stream_ptr(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(getattr(stream, "cuda_stream", stream))


def usr_eval(ctx: int, n: int, xyzq_ptr: int, out_ptr: int, energy_ptr: Optional[int], stream=None):
    _check(lib().usr_eval(ctx, int(n), xyzq_ptr, out_ptr, energy_ptr, _stream_ptr(stream)), "usr_eval")


def usr_eval_host(ctx: int, n: int, xyzq_ptr: int, out_ptr: int, energy_ptr: Optional[int], stream=None):
    _check(lib().usr_eval_host(ctx, int(n), xyzq_ptr, out_ptr, energy_ptr, _stream_ptr(stream)), "usr_eval_host")


def usr_eval_host_async(ctx: int, n: int, xyzq_ptr: int, out_ptr: int, energy_ptr: Optional[int], stream=None):
    _check(lib().usr_eval_host_async(ctx, int(n), xyzq_ptr, out_ptr, energy_ptr, _stream_ptr(stream)),
           "usr_eval_host_async")


def usr_last_device_status(ctx: int) -> int:
    return lib().usr_last_device_status(ctx)


def usr_debug_cells(ctx, n, xyzq_ptr, cell_ptr, perm_ptr, start_ptr, xw_ptr, stream=None):
    _check(lib().usr_debug_cells(ctx, int(n), xyzq_ptr, cell_ptr, perm_ptr, start_ptr, xw_ptr,
                                 _stream_ptr(stream)), "usr_debug_cells")


def usr_debug_pairs(ctx, n, xyzq_ptr, count_ptr, hash_ptr, stream=None):
    _check(lib().usr_debug_pairs(ctx, int(n), xyzq_ptr, count_ptr, hash_ptr, _stream_ptr(stream)), "usr_debug_pairs")


def usr_cells_static(n, xyzq_ptr, box, cells, cell_ptr, perm_ptr, start_ptr, xw_ptr, stream=None):
    b = (_c_d * 3)(*[float(v) for v in box])
    c = (_c_i * 3)(*[int(v) for v in cells])
    _check(lib().usr_cells_static(int(n), xyzq_ptr, b, c, cell_ptr, perm_ptr, start_ptr, xw_ptr,
                                  _stream_ptr(stream)), "usr_cells_static")


def usr_virial(ctx, W_ptr, stream=None):
    _check(lib().usr_virial(ctx, W_ptr, _stream_ptr(stream)), "usr_virial")


def usr_net_charge(ctx, q_ptr, stream=None):
    _check(lib().usr_net_charge(ctx, q_ptr, _stream_ptr(stream)), "usr_net_charge")


def usr_server_create(hbm_budget_bytes=0.0, slots=0) -> int:
    p = usr_server_params(float(hbm_budget_bytes), int(slots))
    h = _c_p()
    _check(lib().usr_server_create(ctypes.byref(p), ctypes.byref(h)), "usr_server_create")
    return h.value


def usr_server_submit(server, params: usr_params, n: int, xyzq_ptr: int, out_ptr: int,
                      energy_ptr: Optional[int]) -> int:
    t = ctypes.c_longlong(0)
    _check(lib().usr_server_submit(server, ctypes.byref(params), int(n), xyzq_ptr, out_ptr, energy_ptr,
                                   ctypes.byref(t)), "usr_server_submit")
    return t.value


def usr_server_poll(server, max_n: int = 1024):
    """Completed requests as (ticket, latency_ms, status) tuples (at most max_n)."""
    if max_n <= 0:
        return []
    tk = (ctypes.c_longlong * max_n)()
    lat = (_c_d * max_n)()
    st = (_c_i * max_n)()
    k = lib().usr_server_poll(server, tk, lat, st, int(max_n))
    return [(int(tk[i]), float(lat[i]), int(st[i])) for i in range(k)]


def usr_server_wait(server, timeout_s: float = 0.0):
    _check(lib().usr_server_wait(server, float(timeout_s)), "usr_server_wait")


def usr_server_info(server) -> Tuple[float, int, int]:
    """(device bytes the slots hold, requests waiting for admission, requests on the device)."""
    b = _c_d(0.0)
    q = ctypes.c_longlong(0)
    f = ctypes.c_longlong(0)
    _check(lib().usr_server_info(server, ctypes.byref(b), ctypes.byref(q), ctypes.byref(f)), "usr_server_info")
    return float(b.value), int(q.value), int(f.value)


def usr_server_destroy(server):
    lib().usr_server_destroy(server)


def usr_set_keep_parts(ctx, on: bool):
    _check(lib().usr_set_keep_parts(ctx, int(bool(on))), "usr_set_keep_parts")


def usr_debug_parts(ctx, near_ptr, far_ptr, stream=None):
    _check(lib().usr_debug_parts(ctx, near_ptr, far_ptr, _stream_ptr(stream)), "usr_debug_parts")


def usr_debug_inject_timeout(ctx, on: bool):
    _check(lib().usr_debug_inject_timeout(ctx, int(bool(on))), "usr_debug_inject_timeout")


def usr_fp32_peak() -> float:
    """Measured FP32 FMA throughput of the current device (TFLOP/s)."""
    v = _c_d(0.0)
    _check(lib().usr_fp32_peak(ctypes.byref(v)), "usr_fp32_peak")
    return float(v.value)


def usr_set_profiling(ctx, on):
    """on: True or 1 every stage boundary, 2 the pair kernel only, False or 0 none."""
    _check(lib().usr_set_profiling(ctx, int(on)), "usr_set_profiling")


def usr_stage_times(ctx) -> Tuple[float, ...]:
    ms = (ctypes.c_float * USR_NSTAGES)()
    _check(lib().usr_stage_times(ctx, ms), "usr_stage_times")
    return tuple(float(v) for v in ms)


def _require(t, name: str, cuda: bool, dtype: str, min_numel: int = 0, rows4: bool = False):
    """Refuse (ValueError) a tensor whose data pointer the library must not be given: not a torch tensor, on
    the wrong side (device / host), of the wrong dtype, not contiguous, or too small.  rows4: an (n, 4)
    matrix.  Checked before any library call, so that a wrong buffer never reaches a copy or a kernel."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name}: a torch tensor is required")
    if t.is_cuda != cuda:
        raise ValueError(f"{name}: a {'CUDA' if cuda else 'host'} tensor is required")
    if t.dtype != getattr(torch, dtype):
        raise ValueError(f"{name}: dtype {dtype} is required, not {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: a contiguous tensor is required")
    if rows4 and (t.dim() != 2 or t.shape[1] != 4):
        raise ValueError(f"{name}: shape (n, 4) is required, not {tuple(t.shape)}")
    if t.numel() < min_numel:
        raise ValueError(f"{name}: at least {min_numel} elements are required, not {t.numel()}")


def _same_device(*ts):
    devs = {t.device for t in ts}
    if len(devs) != 1:
        raise ValueError(f"tensors on different devices: {sorted(str(d) for d in devs)}")


class USeries:
    """One evaluation context (a usr_ctx) with torch-tensor conveniences.

    xyzq: (n, 4) float32 CUDA tensor of (x, y, z, q); results are (n, 4)
    float32 (Fx, Fy, Fz, phi) and a float64 tensor (E, E_near, E_far, E_self).
    """

    def __init__(self, box, grid, r_c, series="C1_B2", max_atoms=0, **kw):
        self.params = make_params(box, grid, r_c, series, max_atoms=max_atoms, **kw)
        self.ctx = usr_init(self.params)
        self.info = usr_info(self.ctx)
        self.max_atoms = max_atoms
        self._last_n = None           # rows of the last evaluation made through this object

    def reconfigure(self, box, grid, r_c, series="C1_B2", max_atoms=0, stream=None, **kw):
        """Point this context at another system (usr_reconfigure)."""
        self.params = make_params(box, grid, r_c, series, max_atoms=max_atoms, **kw)
        usr_reconfigure(self.ctx, self.params, stream)
        self.info = usr_info(self.ctx)
        self.max_atoms = max_atoms
        self._last_n = None

    def close(self):
        if self.ctx:
            usr_destroy(self.ctx)
            self.ctx = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def eval(self, xyzq, out=None, energy=None, stream=None):
        import torch
        _require(xyzq, "xyzq", cuda=True, dtype="float32", rows4=True)
        n = xyzq.shape[0]
        if out is not None:
            _require(out, "out", cuda=True, dtype="float32", min_numel=4 * n)
        if energy is not None:
            _require(energy, "energy", cuda=True, dtype="float64", min_numel=4)
        if out is None:
            out = torch.empty((n, 4), dtype=torch.float32, device=xyzq.device)
        if energy is None:
            energy = torch.empty(4, dtype=torch.float64, device=xyzq.device)
        _same_device(xyzq, out, energy)
        usr_eval(self.ctx, n, xyzq.data_ptr(), out.data_ptr(), energy.data_ptr(), stream)
        self._last_n = n
        return out, energy

    def eval_host(self, xyzq, out=None, energy=None, stream=None):
        """xyzq: (n, 4) float32 host tensor (pinned for asynchronous copies)."""
        import torch
        _require(xyzq, "xyzq", cuda=False, dtype="float32", rows4=True)
        n = xyzq.shape[0]
        if out is not None:
            _require(out, "out", cuda=False, dtype="float32", min_numel=4 * n)
        if energy is not None:
            _require(energy, "energy", cuda=False, dtype="float64", min_numel=4)
        if out is None:
            out = torch.empty((n, 4), dtype=torch.float32, pin_memory=True)
        if energy is None:
            energy = torch.empty(4, dtype=torch.float64, pin_memory=True)
        usr_eval_host(self.ctx, n, xyzq.data_ptr(), out.data_ptr(), energy.data_ptr(), stream)
        self._last_n = n
        return out, energy

    def virial(self):
        """3 x 3 float64 CUDA tensor: the virial of the last evaluation (virial=1 contexts)."""
        import torch
        W = torch.empty(9, dtype=torch.float64, device="cuda")
        usr_virial(self.ctx, W.data_ptr())
        return W.view(3, 3)

    def net_charge(self, stream=None) -> float:
        """Net charge sum q of the last evaluation, as summed on the GPU (synchronises the device)."""
        import torch
        q = torch.empty(1, dtype=torch.float64, pin_memory=True)
        usr_net_charge(self.ctx, q.data_ptr(), stream)
        torch.cuda.synchronize()
        return float(q[0])

    def debug_cells(self, xyzq, stream=None):
        import torch
        _require(xyzq, "xyzq", cuda=True, dtype="float32", rows4=True)
        n = xyzq.shape[0]
        ncell = self.info.cells[0] * self.info.cells[1] * self.info.cells[2]
        dev = xyzq.device
        cell = torch.empty(n, dtype=torch.int32, device=dev)
        perm = torch.empty(n, dtype=torch.int32, device=dev)
        start = torch.empty(ncell + 1, dtype=torch.int32, device=dev)
        xw = torch.empty((n, 4), dtype=torch.float32, device=dev)
        usr_debug_cells(self.ctx, n, xyzq.data_ptr(), cell.data_ptr(), perm.data_ptr(), start.data_ptr(),
                        xw.data_ptr(), stream)
        return cell, perm, start, xw

    def debug_pairs(self, xyzq):
        import torch
        _require(xyzq, "xyzq", cuda=True, dtype="float32", rows4=True)
        n = xyzq.shape[0]
        count = torch.empty(n, dtype=torch.int32, device=xyzq.device)
        h = torch.empty(n, dtype=torch.int64, device=xyzq.device)
        usr_debug_pairs(self.ctx, n, xyzq.data_ptr(), count.data_ptr(), h.data_ptr())
        return count, h

    def parts(self, n):
        """Near and far parts of the last evaluation, which had n rows (the library copies that many)."""
        import torch
        if n != self._last_n:
            raise ValueError(f"parts({n}): the last evaluation through this object had {self._last_n} rows")
        near = torch.empty((n, 4), dtype=torch.float32, device="cuda")
        far = torch.empty((n, 4), dtype=torch.float32, device="cuda")
        usr_debug_parts(self.ctx, near.data_ptr(), far.data_ptr())
        return near, far


class Server:
    """Continuous-batching server (usr_server_*): independent systems evaluated
    as they arrive, up to `slots` at once within `hbm_budget_bytes`.

    submit() takes pinned host tensors and keeps them referenced until the
    request completes; poll() returns (ticket, latency_ms, status) tuples.
    """

    def __init__(self, hbm_budget_bytes=0.0, slots=0):
        self.handle = usr_server_create(hbm_budget_bytes, slots)
        self._live = {}

    def submit(self, params: usr_params, xyzq, out, energy=None) -> int:
        _require(xyzq, "xyzq", cuda=False, dtype="float32", rows4=True)
        n = int(xyzq.shape[0])
        _require(out, "out", cuda=False, dtype="float32", min_numel=4 * n)
        if energy is not None:
            _require(energy, "energy", cuda=False, dtype="float64", min_numel=4)
        t = usr_server_submit(self.handle, params, n, xyzq.data_ptr(), out.data_ptr(),
                              energy.data_ptr() if energy is not None else None)
        self._live[t] = (params, xyzq, out, energy)
        return t

    def poll(self, max_n=1024):
        res = usr_server_poll(self.handle, max_n)
        for tk, _, _ in res:
            self._live.pop(tk, None)
        return res

    def wait(self, timeout_s=0.0):
        usr_server_wait(self.handle, timeout_s)

    def info(self):
        return usr_server_info(self.handle)

    def close(self):
        if self.handle:
            usr_server_destroy(self.handle)
            self.handle = 0
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
