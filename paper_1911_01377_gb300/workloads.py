"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no u-series arithmetic: it only draws charges and positions,
so both the GPU library and the FP64 oracle can be fed the same numbers.  All
generators work in float64 and round once to float32 at the end; the rounded
values are what both sides see.

Water model: rigid 3-site water, O -0.834 e, two H +0.417 e at 0.9572 A with
an H-O-H angle of 104.52 degrees, uniformly random orientation (random unit
quaternion), O centres placed by random sequential addition with O-O >= 2.5 A
under periodic boundaries.  The paper's DPPC configurations are not available;
the membrane-slab workload stands in for its lipid bilayer (72 DPPC + 2189
waters, Sec. IV): a 40 A slab of chain-like beads between two water layers.
"""
from __future__ import annotations

import hashlib
import math
import os
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

import numpy as np

SEED_BASE = 191101377

Q_O = -0.834
Q_H = 0.417
R_OH = 0.9572
THETA_HOH = math.radians(104.52)
WATER_DENSITY = 0.1 / 3.0   # waters per A^3 (0.1 charges per A^3)


@dataclass
class Workload:
    """One evaluation problem: box (A), grid points per axis, cutoffs, charges."""
    name: str
    box: Tuple[float, float, float]
    grid: Tuple[int, int, int]
    r_c: Tuple[float, ...]
    xyzq: np.ndarray                      # (N, 4) float32: x, y, z, q
    description: str = ""
    meta: Dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.xyzq.shape[0])


def random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniformly distributed rotation matrices from random unit quaternions (Shoemake)."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a = np.sqrt(1.0 - u1) * np.sin(2 * np.pi * u2)
    b = np.sqrt(1.0 - u1) * np.cos(2 * np.pi * u2)
    c = np.sqrt(u1) * np.sin(2 * np.pi * u3)
    d = np.sqrt(u1) * np.cos(2 * np.pi * u3)
    # quaternion (w, x, y, z) = (d, a, b, c)
    w, x, y, z = d, a, b, c
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


class _Hash:
    """Periodic cell hash of accepted points for hard-core rejection tests."""

    def __init__(self, box, cell_min: float, cap: int = 16):
        self.box = np.asarray(box, dtype=np.float64)
        self.nc = np.maximum(1, np.floor(self.box / cell_min).astype(np.int64))
        self.cs = self.box / self.nc
        self.cap = cap
        self.idx = -np.ones((int(np.prod(self.nc)), cap), dtype=np.int64)
        self.fill = np.zeros(int(np.prod(self.nc)), dtype=np.int64)
        self.pts = np.zeros((0, 3))
        self._buf = np.zeros((1024, 3))
        self.count = 0

    def _cell3(self, p):
        c = np.floor(np.mod(p, self.box) / self.cs).astype(np.int64)
        return np.minimum(c, self.nc - 1)

    def _lin(self, c3):
        return (c3[..., 2] * self.nc[1] + c3[..., 1]) * self.nc[0] + c3[..., 0]

    _OFFS = np.array([[ox, oy, oz] for oz in (-1, 0, 1) for oy in (-1, 0, 1) for ox in (-1, 0, 1)])

    def min_dist2(self, p: np.ndarray) -> np.ndarray:
        """Squared periodic distance from each row of p to its nearest stored point."""
        p = np.atleast_2d(p)
        if self.count == 0:
            return np.full(p.shape[0], np.inf)
        c3 = self._cell3(p)
        nb = self._lin(np.mod(c3[:, None, :] + self._OFFS[None, :, :], self.nc))   # (m, 27)
        mf = max(1, int(self.fill.max()))                   # slots in use in the fullest cell
        ids = self.idx[nb, :mf].reshape(p.shape[0], -1)                             # (m, 27 mf)
        valid = ids >= 0
        q = self._buf[np.where(valid, ids, 0)]                                      # (m, 27 cap, 3)
        d = q - p[:, None, :]
        d -= self.box * np.round(d / self.box)
        r2 = np.where(valid, np.sum(d * d, axis=-1), np.inf)
        return r2.min(axis=1)

    def add(self, p: np.ndarray):
        p = np.atleast_2d(p)
        need = self.count + p.shape[0]
        if need > self._buf.shape[0]:
            nb = np.zeros((max(need, 2 * self._buf.shape[0]), 3))
            nb[: self.count] = self._buf[: self.count]
            self._buf = nb
        lin = self._lin(self._cell3(p))
        for k in range(p.shape[0]):
            c = lin[k]
            if self.fill[c] >= self.cap:
                raise RuntimeError("hash cell overflow")
            self.idx[c, self.fill[c]] = self.count
            self.fill[c] += 1
            self._buf[self.count] = p[k]
            self.count += 1


def _rsa_centres(rng, box, n, dmin, zrange=None, avoid: Optional[_Hash] = None,
                 avoid_d: float = 1.0, site_fn=None, batch: int = 512, max_batches: int = 200000):
    """Random sequential addition of n centres with periodic minimum separation dmin.

    zrange: optional (z0, length) -- centres drawn with z in [z0, z0+length) mod Lz.
    avoid / avoid_d / site_fn: every site returned by site_fn(centres) must lie at
    least avoid_d from the points already stored in `avoid`.
    """
    box = np.asarray(box, dtype=np.float64)
    H = _Hash(box, dmin, cap=8)
    out = np.zeros((n, 3))
    extra = []
    got = 0
    d2 = dmin * dmin
    for _ in range(max_batches):
        if got >= n:
            break
        c = rng.random((batch, 3)) * box
        if zrange is not None:
            c[:, 2] = np.mod(zrange[0] + rng.random(batch) * zrange[1], box[2])
        ok = H.min_dist2(c) >= d2
        payload = None
        if site_fn is not None:
            payload = site_fn(c)
            if avoid is not None and ok.any():
                sites = payload[0]                         # (batch, s, 3)
                md = avoid.min_dist2(sites.reshape(-1, 3)).reshape(sites.shape[0], -1)
                ok &= np.all(md >= avoid_d * avoid_d, axis=1)
        # greedy acceptance within the batch: candidates that passed against the
        # stored points only need checking against earlier accepted candidates
        cand = np.nonzero(ok)[0]
        if cand.size == 0:
            continue
        d = c[cand][:, None, :] - c[cand][None, :, :]
        d -= box * np.round(d / box)
        clash = np.sum(d * d, axis=-1) < d2
        keep = np.zeros(cand.size, dtype=bool)
        for a in range(cand.size):
            if got + int(keep.sum()) >= n:
                break
            if not np.any(clash[a, :a] & keep[:a]):
                keep[a] = True
        acc = cand[keep]
        H.add(c[acc])
        out[got:got + acc.size] = c[acc]
        if payload is not None:
            extra.extend(tuple(x[k] for x in payload) for k in acc)
        got += acc.size
    if got < n:
        raise RuntimeError(f"random sequential addition stalled at {got}/{n}")
    return out, extra


def _water_sites(rng):
    """site_fn for waters: returns (sites (b,3,3), charges (b,3))."""
    local = np.array([[0.0, 0.0, 0.0],
                      [R_OH * math.sin(THETA_HOH / 2), 0.0, R_OH * math.cos(THETA_HOH / 2)],
                      [-R_OH * math.sin(THETA_HOH / 2), 0.0, R_OH * math.cos(THETA_HOH / 2)]])

    def fn(c):
        R = random_rotations(rng, c.shape[0])
        sites = c[:, None, :] + np.einsum("bij,sj->bsi", R, local)
        return (sites,)
    return fn


def water_box(seed: int, box, n_waters: int, zrange=None, avoid: Optional[_Hash] = None) -> np.ndarray:
    """(3 n_waters, 4) float64 rows x, y, z, q: O then its two H, per water."""
    rng = np.random.default_rng(seed)
    _, extra = _rsa_centres(rng, box, n_waters, 2.5, zrange=zrange, avoid=avoid,
                            site_fn=_water_sites(rng))
    sites = np.stack([e[0] for e in extra])                # (n, 3, 3)
    q = np.tile(np.array([Q_O, Q_H, Q_H]), (n_waters, 1))
    return np.concatenate([sites.reshape(-1, 3), q.reshape(-1, 1)], axis=1)


def _finish(name, box, grid, r_c, rows, description, **meta) -> Workload:
    xyzq = np.ascontiguousarray(rows.astype(np.float32))
    return Workload(name, tuple(float(v) for v in box), tuple(int(v) for v in grid),
                    tuple(float(v) for v in r_c), xyzq, description, meta)


def _disk_cached(name: str, make) -> np.ndarray:
    """Rows of a large generated workload, kept in _cache/ next to this file under a
    key that changes with this file's source (a generator change regenerates)."""
    with open(__file__, "rb") as f:
        key = hashlib.sha1(f.read()).hexdigest()[:16]
    d = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_cache")
    path = os.path.join(d, f"{name}-{key}.npy")
    if os.path.exists(path):
        return np.load(path)
    rows = make()
    os.makedirs(d, exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "wb") as f:
        np.save(f, rows)
    os.replace(tmp, path)
    return rows


def water_workload(index: int, name: str, n_waters: int, L: float, r_c, grid) -> Workload:
    def make():
        return water_box(SEED_BASE + index, (L, L, L), n_waters)
    rows = _disk_cached(name, make) if n_waters > 100000 else make()
    return _finish(name, (L, L, L), grid, r_c, rows,
                   f"{n_waters} rigid 3-site waters ({3 * n_waters} charges), cubic box L={L} A")


def membrane_slab(index: int = 1, box=(80.0, 80.0, 100.0), slab=(30.0, 70.0), chains: int = 2133,
                  beads: int = 12, n_waters: int = 12800, r_c=(8.0, 9.0, 10.0, 11.0, 12.0, 13.0),
                  grid=(64, 64, 80)) -> Workload:
    """Lipid-membrane-shaped slab: chain-like beads in z in [30, 70] A, waters outside.

    Beads: random walks of 12 beads with 1.53 A bonds, each bead >= 1.0 A from
    every other bead, chains of the lower leaflet start near z = 30 A and walk
    toward +z, those of the upper leaflet start near z = 70 A and walk toward -z.
    Bead charges are N(0, 0.3 e), shifted per 12-bead chain to zero net charge.
    Waters: O centres with z outside the slab, every water site >= 1.0 A from
    every bead.
    """
    rng = np.random.default_rng(SEED_BASE + index)
    box = np.asarray(box, dtype=np.float64)
    z0, z1 = slab
    zmid = 0.5 * (z0 + z1)
    BH = _Hash(box, 1.0, cap=8)
    bead_pos = np.zeros((chains * beads, 3))
    bond = 1.53
    k = 0
    for c in range(chains):
        lower = c % 2 == 0
        direction = 1.0 if lower else -1.0
        lo, hi = (z0, zmid) if lower else (zmid, z1)
        for attempt in range(5000):
            start = np.array([rng.random() * box[0], rng.random() * box[1],
                              (z0 + 1.0 + rng.random() * 9.0) if lower else (z1 - 1.0 - rng.random() * 9.0)])
            chain = [start]
            ok = BH.min_dist2(start)[0] >= 1.0
            while ok and len(chain) < beads:
                # 8 proposed bond directions at once; the first admissible one is taken
                u = rng.normal(size=(8, 3))
                u /= np.linalg.norm(u, axis=1, keepdims=True)
                u[:, 2] += 0.6 * direction
                u /= np.linalg.norm(u, axis=1, keepdims=True)
                p = chain[-1] + bond * u
                good = (p[:, 2] >= lo) & (p[:, 2] < hi)
                good &= BH.min_dist2(p) >= 1.0
                own = np.array(chain[:-1]) if len(chain) > 1 else np.zeros((0, 3))
                if own.shape[0]:
                    dd = np.sum((p[:, None, :] - own[None, :, :]) ** 2, axis=-1)
                    good &= np.all(dd >= 1.0, axis=1)
                idx = np.nonzero(good)[0]
                ok = idx.size > 0
                if ok:
                    chain.append(p[idx[0]])
            if ok:
                break
        else:
            raise RuntimeError("chain growth stalled")
        pts = np.array(chain)
        pts[:, :2] = np.mod(pts[:, :2], box[:2])
        BH.add(pts)
        bead_pos[k:k + beads] = pts
        k += beads
    qb = _quantised_neutral(rng.normal(0.0, 0.3, size=(chains, beads)))
    beads_rows = np.concatenate([bead_pos, qb.reshape(-1, 1)], axis=1)
    # waters: O in z outside [z0, z1) (periodic), sites >= 1 A from beads
    wrows = water_box(SEED_BASE + 100 + index, tuple(box), n_waters,
                      zrange=(z1, box[2] - (z1 - z0)), avoid=BH)
    rows = np.concatenate([beads_rows, wrows], axis=0)
    return _finish("membrane_slab_64k", tuple(box), grid, r_c, rows,
                   f"membrane-shaped slab {box[0]:g}x{box[1]:g}x{box[2]:g} A: {chains}x{beads} beads "
                   f"in z=[{z0:g},{z1:g}] A + {n_waters} waters ({rows.shape[0]} charges)",
                   n_beads=chains * beads, n_waters=n_waters)


def _quantised_neutral(q: np.ndarray) -> np.ndarray:
    """Shift each row to zero mean, round to multiples of 2^-20 (exact in float32)
    and fix the last entry so that every row sums to exactly zero."""
    q = q - q.mean(axis=1, keepdims=True)
    q = np.round(q * 2.0 ** 20) / 2.0 ** 20
    q[:, -1] = -q[:, :-1].sum(axis=1)
    return q


_CACHE: Dict[str, Workload] = {}


def get(name: str) -> Workload:
    """Named workloads:
      water_3k        1,000 waters, L = 31.0 A, r_c = 9 A, 32^3 grid (small parity case)
      membrane_slab   ~64,000 charges, 80x80x100 A, r_c = 8..13 A, 64x64x80 grid
      water_20k       6,667 waters (20,001 charges), L = 58.5 A, r_c = 9 A, 48^3 grid
      water_1m        354,933 waters (1,064,799 charges), L = 220 A, r_c = 10 A, 176^3 grid
    """
    if name in _CACHE:
        return _CACHE[name]
    if name == "water_3k":
        w = water_workload(0, name, 1000, 31.0, (9.0,), (32, 32, 32))
    elif name == "membrane_slab":
        w = membrane_slab(1)
    elif name == "water_1m":
        w = water_workload(2, name, 354933, 220.0, (10.0,), (176, 176, 176))
    elif name == "water_20k":
        w = water_workload(3, name, 6667, 58.5, (9.0,), (48, 48, 48))
    else:
        raise KeyError(name)
    _CACHE[name] = w
    return w


def lattice_water_box(seed: int, n_charges: int, density: float = 0.1) -> Tuple[Tuple[float, float, float], np.ndarray]:
    """A cubic water box of n_charges (a multiple of 3) at `density` charges per A^3,
    generated fast for serving streams: O centres on randomly chosen sites of a
    periodic cubic lattice (spacing ~3.1 A at water density) with a jitter of at
    most 0.25 A per axis, so that O-O distances stay >= 2.5 A without rejection;
    uniformly random orientations.  Returns (box, xyzq)."""
    rng = np.random.default_rng(seed)
    n_w = n_charges // 3
    L = (3 * n_w / density) ** (1.0 / 3.0)
    m = int(math.ceil(n_w ** (1.0 / 3.0) - 1e-9))
    a = L / m
    if a < 2.5:
        raise ValueError("lattice too dense for the O-O separation")
    jit = min(0.25, 0.5 * (a - 2.5))            # keeps O-O >= 2.5 A
    sites = rng.choice(m ** 3, size=n_w, replace=False)
    iz, rem = np.divmod(sites, m * m)
    iy, ix = np.divmod(rem, m)
    centres = (np.stack([ix, iy, iz], axis=1) + 0.5) * a + rng.uniform(-jit, jit, size=(n_w, 3))
    R = random_rotations(rng, n_w)
    half = 0.5 * THETA_HOH
    local = np.array([[0.0, 0.0, 0.0],
                      [R_OH * math.sin(half), 0.0, R_OH * math.cos(half)],
                      [-R_OH * math.sin(half), 0.0, R_OH * math.cos(half)]])
    sites_xyz = centres[:, None, :] + np.einsum("nij,kj->nki", R, local)
    q = np.tile(np.array([Q_O, Q_H, Q_H]), (n_w, 1))
    rows = np.concatenate([sites_xyz.reshape(-1, 3), q.reshape(-1, 1)], axis=1)
    return (L, L, L), np.ascontiguousarray(rows.astype(np.float32))


# The serving stream's evaluation form: TF32x3 tensor-core convolutions and a 10-point spreading stencil of
# width 0.9 h.  On the stream's lattice-placed boxes (~1 A grids, r_c = 9 A) the grid errors of the ordered
# charges add up coherently: the 8-point stencil (width 0.83 h) leaves about 1.2e-4 of the far potential and
# single-grid BF16x3 about 6e-4 (the wide terms' near-constant parts carry the 16-bit split's rounding), against
# 6-7e-5 for randomly placed waters; this form stays near 2e-5 on the lattice boxes.
SERVING_FORM = dict(conv=1, spread_points=10, spread_sigma_over_h=0.9)


def serving_stream(seed: int, count: int, n_min: int = 2000, n_max: int = 200000, density: float = 0.1,
                   spacing: float = 1.0, r_c: float = 9.0, grid_multiple: int = 8):
    """The serving workload: `count` independent water boxes with charge counts
    log-uniform in [n_min, n_max] (multiples of 3), cubic boxes sized to the
    density, grids of about `spacing` A rounded to a multiple of grid_multiple.
    Yields (box, grid, r_c, xyzq) lazily (generation is the slow part)."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(math.log(n_min), math.log(n_max), size=count))
    for k, nf in enumerate(ns):
        n = max(3, int(round(nf / 3.0)) * 3)
        box, xyzq = lattice_water_box(seed * 1000 + k, n, density)
        g = max(grid_multiple * 3, int(round(box[0] / spacing / grid_multiple)) * grid_multiple)
        yield box, (g, g, g), r_c, xyzq


def random_neutral(seed: int, n: int, box, qscale: float = 1.0, min_dist: float = 0.0) -> np.ndarray:
    """n random charges (float32 rows) in a box, charges shifted to sum to zero."""
    rng = np.random.default_rng(seed)
    box = np.asarray(box, dtype=np.float64)
    if min_dist > 0:
        pos, _ = _rsa_centres(rng, box, n, min_dist, batch=64)
    else:
        pos = rng.random((n, 3)) * box
    q = _quantised_neutral(rng.normal(0.0, qscale, size=(1, n))).reshape(-1)
    return np.concatenate([pos, q[:, None]], axis=1).astype(np.float32)
