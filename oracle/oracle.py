"""ctypes binding of the FP64 oracle (oracle/usr_oracle.c).  Test infrastructure only.

Every routine takes the u-series parameters (b, r0, w0, s0) of Eqs. 24/28 and
the cutoff r_c; sigma = r_c / r0 (Eq. 23).  Positions are (N, 3) arrays in
Angstrom, charges (N,) in e; single-precision inputs are promoted exactly to
double before use, so the oracle sees the same numbers as the GPU.
"""
from __future__ import annotations

import ctypes
import os
from typing import NamedTuple, Optional

import numpy as np

from . import build as _build

_lib = None

_d = ctypes.c_double
_i = ctypes.c_int
_pd = ctypes.POINTER(ctypes.c_double)
_pi = ctypes.POINTER(ctypes.c_int)
_pf = ctypes.POINTER(ctypes.c_float)
_pu64 = ctypes.POINTER(ctypes.c_uint64)


class Series(NamedTuple):
    """Parameters of one u-series construction (Tables 1 and 2)."""
    b: float
    r0: float
    w0: float
    s0: float = 1.0


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        sp = [_d, _d, _d, _d, _d]
        L.or_num_terms.argtypes = sp
        L.or_num_terms.restype = _i
        L.or_terms_table.argtypes = sp + [_i, _pd, _pd]
        L.or_terms_table.restype = _i
        L.or_far_function.argtypes = sp + [_i, _pd, _pd, _pd]
        L.or_far_fhat.argtypes = sp + [_i, _i, _pd, _pd]
        L.or_F0.argtypes = sp
        L.or_F0.restype = _d
        L.or_near.argtypes = sp + [_pd, _i, _pd, _pd, _i, _pi, _pd, _pd]
        L.or_near.restype = _i
        L.or_far.argtypes = sp + [_pd, _i, _d, _i, _pd, _pd, _i, _pi, _pd, _pd, _pd, _pi]
        L.or_far.restype = _i
        L.or_far_realspace.argtypes = sp + [_pd, _i, _i, _pd, _pd, _pd, _pd, _pd]
        L.or_far_realspace.restype = _i
        L.or_eval.argtypes = sp + [_pd, _i, _d, _i, _pd, _pd, _i, _pi, _pd, _pd, _pd, _pd, _pd, _pd, _pd]
        L.or_eval.restype = _i
        L.or_virial.argtypes = sp + [_pd, _i, _d, _i, _pd, _pd, _pd, _pd]
        L.or_virial.restype = _i
        L.or_far_virial_realspace.argtypes = sp + [_pd, _i, _i, _pd, _pd, _pd]
        L.or_far_virial_realspace.restype = _i
        L.or_ewald.argtypes = [_pd, _d, _d, _d, _i, _pd, _pd, _pd, _pd, _pd]
        L.or_ewald.restype = _i
        L.or_canon_cells.argtypes = [_i, _pf, _pd, _pi, _pi, _pf]
        L.or_canon_pairs.argtypes = [_i, _pf, _pd, _pi, _d, _pi, _pu64]
        L.or_canon_pairs.restype = _i
        L.or_num_threads.restype = _i
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_pd)


def _prep(box, pos, q):
    box = np.ascontiguousarray(np.asarray(box, dtype=np.float64).reshape(3))
    pos = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(-1, 3))
    q = np.ascontiguousarray(np.asarray(q, dtype=np.float64).reshape(-1))
    assert pos.shape[0] == q.shape[0]
    return box, pos, q


def _targets(targets, n):
    if targets is None:
        return None, n, None
    t = np.ascontiguousarray(np.asarray(targets, dtype=np.int32).reshape(-1))
    assert t.size == 0 or (t.min() >= 0 and t.max() < n)
    return t, t.size, t.ctypes.data_as(_pi)


def num_threads() -> int:
    return lib().or_num_threads()


def terms(series: Series, r_c: float, nmax: int = 4096):
    """(a_j, s_j) of the far series, Eqs. 19/24/28 with sigma = r_c / r0."""
    a = np.zeros(nmax)
    s = np.zeros(nmax)
    n = lib().or_terms_table(*series, r_c, nmax, _dp(a), _dp(s))
    n = min(n, nmax)
    return a[:n].copy(), s[:n].copy()


def far_function(series: Series, r_c: float, r):
    """F(r) and F'(r)/r of the full far series."""
    r = np.ascontiguousarray(np.asarray(r, dtype=np.float64).reshape(-1))
    F = np.zeros_like(r)
    G = np.zeros_like(r)
    lib().or_far_function(*series, r_c, r.size, _dp(r), _dp(F), _dp(G))
    return F, G


def far_fhat(series: Series, r_c: float, k, n_terms: int = 0):
    k = np.ascontiguousarray(np.asarray(k, dtype=np.float64).reshape(-1))
    out = np.zeros_like(k)
    lib().or_far_fhat(*series, r_c, n_terms, k.size, _dp(k), _dp(out))
    return out


def F0(series: Series, r_c: float) -> float:
    """F(0) of the full series (self-interaction constant)."""
    return lib().or_F0(*series, r_c)


def near(series: Series, r_c, box, pos, q, targets=None):
    box, pos, q = _prep(box, pos, q)
    t, nt, tp = _targets(targets, q.size)
    phi = np.zeros(nt)
    f = np.zeros((nt, 3))
    rc = lib().or_near(*series, r_c, _dp(box), q.size, _dp(pos), _dp(q), nt, tp, _dp(phi), _dp(f))
    assert rc == 0
    return phi, f


def far(series: Series, r_c, box, pos, q, targets=None, n_terms: int = 0, kmax: float = 0.0):
    """Exact k-space far part; returns (E_far, phi_far, f_far, number of half-space k)."""
    box, pos, q = _prep(box, pos, q)
    t, nt, tp = _targets(targets, q.size)
    phi = np.zeros(nt)
    f = np.zeros((nt, 3))
    e = ctypes.c_double(0.0)
    nk = ctypes.c_int(0)
    rc = lib().or_far(*series, r_c, _dp(box), n_terms, kmax, q.size, _dp(pos), _dp(q), nt, tp,
                      _dp(phi), _dp(f), ctypes.byref(e), ctypes.byref(nk))
    assert rc == 0
    return e.value, phi, f, nk.value


def far_realspace(series: Series, r_c, box, pos, q, n_terms: int):
    box, pos, q = _prep(box, pos, q)
    phi = np.zeros(q.size)
    f = np.zeros((q.size, 3))
    e = ctypes.c_double(0.0)
    rc = lib().or_far_realspace(*series, r_c, _dp(box), n_terms, q.size, _dp(pos), _dp(q),
                                _dp(phi), _dp(f), ctypes.byref(e))
    assert rc == 0
    return e.value, phi, f


class Result(NamedTuple):
    E: float
    E_near: float
    E_far: float
    E_self: float
    phi: np.ndarray
    F: np.ndarray
    phi_near: np.ndarray
    F_near: np.ndarray
    phi_far: np.ndarray
    F_far: np.ndarray


def evaluate(series: Series, r_c, box, pos, q, targets=None, n_terms: int = 0,
             kmax: float = 0.0) -> Result:
    """Full u-series energy, potentials and forces (near + far + self)."""
    box, pos, q = _prep(box, pos, q)
    t, nt, tp = _targets(targets, q.size)
    phi = np.zeros(nt)
    f = np.zeros((nt, 3))
    pn = np.zeros(nt)
    fn = np.zeros((nt, 3))
    pf = np.zeros(nt)
    ff = np.zeros((nt, 3))
    en = np.zeros(4)
    rc = lib().or_eval(*series, r_c, _dp(box), n_terms, kmax, q.size, _dp(pos), _dp(q), nt, tp,
                       _dp(phi), _dp(f), _dp(pn), _dp(fn), _dp(pf), _dp(ff), _dp(en))
    assert rc == 0
    return Result(en[0], en[1], en[2], en[3], phi, f, pn, fn, pf, ff)


def virial(series: Series, r_c, box, pos, q, n_terms: int = 0, kmax: float = 0.0):
    """Virial tensor -dE/d(strain): (W_near, W_far) as 3 x 3 arrays (the self term adds none)."""
    box, pos, q = _prep(box, pos, q)
    wn = np.zeros(9)
    wf = np.zeros(9)
    rc = lib().or_virial(*series, r_c, _dp(box), n_terms, kmax, q.size, _dp(pos), _dp(q), _dp(wn), _dp(wf))
    assert rc == 0
    return wn.reshape(3, 3), wf.reshape(3, 3)


def far_virial_realspace(series: Series, r_c, box, pos, q, n_terms: int):
    """Far-part virial of the first n_terms Gaussians as a real-space image sum (tiny systems)."""
    box, pos, q = _prep(box, pos, q)
    wf = np.zeros(9)
    rc = lib().or_far_virial_realspace(*series, r_c, _dp(box), n_terms, q.size, _dp(pos), _dp(q), _dp(wf))
    assert rc == 0
    return wf.reshape(3, 3)


def ewald(box, pos, q, sigma_e: Optional[float] = None, tol: float = 1e-16):
    """Classic Ewald sum (Eqs. 6-10); returns (E, phi, f)."""
    box, pos, q = _prep(box, pos, q)
    if sigma_e is None:
        sigma_e = min(box) / 6.0
    # erfc(x) < tol at x ~ 5.9 for 1e-16; exp(-s^2 k^2 / 2) < tol at s k ~ 8.6
    rcut = 6.2 * np.sqrt(2.0) * sigma_e
    kmax = 9.0 / sigma_e
    phi = np.zeros(q.size)
    f = np.zeros((q.size, 3))
    en = np.zeros(3)
    rc = lib().or_ewald(_dp(box), sigma_e, rcut, kmax, q.size, _dp(pos), _dp(q), _dp(phi), _dp(f), _dp(en))
    assert rc == 0
    return en[0], phi, f


def canon_cells(xyzq, box, nc):
    """Cell id and wrapped single-precision position per atom (canonical predicate)."""
    xyzq = np.ascontiguousarray(np.asarray(xyzq, dtype=np.float32).reshape(-1, 4))
    box = np.ascontiguousarray(np.asarray(box, dtype=np.float64).reshape(3))
    nc = np.ascontiguousarray(np.asarray(nc, dtype=np.int32).reshape(3))
    n = xyzq.shape[0]
    cell = np.zeros(n, dtype=np.int32)
    xw = np.zeros((n, 3), dtype=np.float32)
    lib().or_canon_cells(n, xyzq.ctypes.data_as(_pf), _dp(box), nc.ctypes.data_as(_pi),
                         cell.ctypes.data_as(_pi), xw.ctypes.data_as(_pf))
    return cell, xw


def canon_pairs(xyzq, box, nc, r_c):
    """Per-atom partner count and order-free hash of the canonical pair list."""
    xyzq = np.ascontiguousarray(np.asarray(xyzq, dtype=np.float32).reshape(-1, 4))
    box = np.ascontiguousarray(np.asarray(box, dtype=np.float64).reshape(3))
    nc = np.ascontiguousarray(np.asarray(nc, dtype=np.int32).reshape(3))
    n = xyzq.shape[0]
    cnt = np.zeros(n, dtype=np.int32)
    h = np.zeros(n, dtype=np.uint64)
    rc = lib().or_canon_pairs(n, xyzq.ctypes.data_as(_pf), _dp(box), nc.ctypes.data_as(_pi), r_c,
                              cnt.ctypes.data_as(_pi), h.ctypes.data_as(_pu64))
    assert rc == 0
    return cnt, h


def rms_rel(a, ref) -> float:
    """sqrt(sum |a - ref|^2 / sum |ref|^2): the ratio-of-norms error measure."""
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = float(np.sum(ref * ref))
    return float(np.sqrt(np.sum((a - ref) ** 2) / den)) if den > 0 else float(np.sqrt(np.sum(a * a)))


__all__ = ["Series", "lib", "num_threads", "terms", "far_function", "far_fhat", "F0", "near", "far",
           "far_realspace", "Result", "evaluate", "ewald", "canon_cells", "canon_pairs", "rms_rel", "virial",
           "far_virial_realspace"]
