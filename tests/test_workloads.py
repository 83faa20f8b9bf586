"""The seeded synthetic inputs follow the stated recipe (no GPU).

Every workload is drawn in float64 and rounded once to float32; both the GPU
library and the oracle see the rounded rows.  These tests check the rounded
rows against the recipe, with tolerances of the float32 rounding of positions
up to 100 A (about 1e-5 A):

  * 3-site waters: O -0.834 e and two H +0.417 e, O-H 0.9572 A, H-O-H 104.52
    degrees, every water exactly neutral, O-O >= 2.5 A under periodic
    boundaries, orientations spread over the sphere;
  * the membrane-shaped slab: 2,133 chains of 12 beads in z in [30, 70) A with
    1.53 A bonds, beads >= 1 A apart, bead charges of spread about 0.3 e made
    exactly neutral per chain, 12,800 waters with O outside the slab and every
    water site >= 1 A from every bead;
  * the serving stream: charge counts multiples of 3, log-uniform in the stated
    range, cubic boxes at 0.1 charges per A^3, grids of about 1 A rounded to a
    multiple of 8;
  * the same seed gives the same bits.
"""
import math

import numpy as np
import pytest

from paper_1911_01377_gb300 import workloads as W

TOL_POS = 2e-5


def _min_image(d, box):
    box = np.asarray(box, dtype=np.float64)
    return d - box * np.round(d / box)


def _periodic_min_dist(points, box):
    """Smallest periodic distance between two distinct rows of points."""
    from scipy.spatial import cKDTree
    box = np.asarray(box, dtype=np.float64)
    p = np.mod(points.astype(np.float64), box)
    p = np.where(p >= box, 0.0, p)
    d, _ = cKDTree(p, boxsize=box).query(p, k=2)
    return float(d[:, 1].min())


def _check_waters(rows, box):
    """rows: (3 m, 4) float32, O then its two H per water."""
    w = rows.reshape(-1, 3, 4).astype(np.float64)
    q = w[:, :, 3]
    assert np.all(q[:, 0] == np.float32(W.Q_O)) and np.all(q[:, 1:] == np.float32(W.Q_H))
    assert np.all(q.sum(axis=1) == 0.0)                       # exactly neutral in float32 arithmetic
    o, h1, h2 = w[:, 0, :3], w[:, 1, :3], w[:, 2, :3]
    r1 = np.linalg.norm(h1 - o, axis=1)
    r2 = np.linalg.norm(h2 - o, axis=1)
    assert np.max(np.abs(r1 - 0.9572)) < TOL_POS and np.max(np.abs(r2 - 0.9572)) < TOL_POS
    cosang = np.sum((h1 - o) * (h2 - o), axis=1) / (r1 * r2)
    ang = np.degrees(np.arccos(np.clip(cosang, -1.0, 1.0)))
    assert np.max(np.abs(ang - 104.52)) < 5e-3
    assert _periodic_min_dist(o, box) >= 2.5 - TOL_POS
    # orientations: the unit dipole directions average to about zero, and each axis carries about a third
    dip = (h1 + h2) * 0.5 - o
    u = dip / np.linalg.norm(dip, axis=1, keepdims=True)
    m = u.shape[0]
    assert np.all(np.abs(u.mean(axis=0)) < 5.0 / math.sqrt(3.0 * m))
    assert np.all(np.abs((u * u).mean(axis=0) - 1.0 / 3.0) < 5.0 * math.sqrt(4.0 / 45.0 / m))
    return o


@pytest.mark.parametrize("name,n_waters,L,grid,r_c", [("water_3k", 1000, 31.0, (32, 32, 32), (9.0,)),
                                                      ("water_20k", 6667, 58.5, (48, 48, 48), (9.0,))])
def test_water_boxes(name, n_waters, L, grid, r_c):
    w = W.get(name)
    assert w.xyzq.dtype == np.float32 and w.xyzq.flags.c_contiguous
    assert w.n == 3 * n_waters and w.box == (L, L, L) and w.grid == grid and w.r_c == r_c
    o = _check_waters(w.xyzq, w.box)
    assert np.all((o >= 0.0) & (o < L + TOL_POS))             # centres drawn in the box (H may stick out)


def test_same_seed_same_bits():
    a = W.water_box(7, (20.0, 20.0, 20.0), 200)
    b = W.water_box(7, (20.0, 20.0, 20.0), 200)
    c = W.water_box(8, (20.0, 20.0, 20.0), 200)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    r1 = W.random_neutral(5, 300, (15.0, 16.0, 17.0), min_dist=1.2)
    r2 = W.random_neutral(5, 300, (15.0, 16.0, 17.0), min_dist=1.2)
    assert np.array_equal(r1, r2)


def test_random_neutral():
    box = (15.0, 16.0, 17.0)
    r = W.random_neutral(11, 500, box, qscale=0.7, min_dist=1.2)
    assert r.dtype == np.float32 and r.shape == (500, 4)
    assert r[:, 3].astype(np.float64).sum() == 0.0
    assert np.all((r[:, :3] >= 0.0) & (r[:, :3] <= np.array(box, dtype=np.float32)))
    assert _periodic_min_dist(r[:, :3], box) >= 1.2 - TOL_POS
    assert 0.5 < r[:, 3].std() < 0.9


def test_membrane_slab():
    w = W.get("membrane_slab")
    box = np.array(w.box)
    assert w.box == (80.0, 80.0, 100.0) and w.grid == (64, 64, 80)
    assert w.r_c == (8.0, 9.0, 10.0, 11.0, 12.0, 13.0)
    nb, nw = w.meta["n_beads"], w.meta["n_waters"]
    assert nb == 2133 * 12 and nw == 12800 and w.n == nb + 3 * nw == 63996
    beads = w.xyzq[:nb].astype(np.float64)
    chains = beads.reshape(2133, 12, 4)
    # beads inside the slab, 1.53 A bonds along each chain (minimum image across the x / y faces)
    assert np.all((beads[:, 2] >= 30.0) & (beads[:, 2] < 70.0))
    bonds = np.linalg.norm(_min_image(np.diff(chains[:, :, :3], axis=1), box), axis=2)
    assert np.max(np.abs(bonds - 1.53)) < TOL_POS
    assert _periodic_min_dist(beads[:, :3], box) >= 1.0 - TOL_POS
    # charges: spread about 0.3 e (0.3 sqrt(11/12) once each chain's mean is removed), each chain neutral
    qb = chains[:, :, 3]
    assert np.all(qb.sum(axis=1) == 0.0)
    assert 0.27 < qb.std() < 0.31
    # the two leaflets: even chains start in the lower half and walk up, odd ones the other way
    assert np.all(chains[0::2, :, 2] < 50.0) and np.all(chains[1::2, :, 2] >= 50.0)
    # waters: O outside the slab, every site at least 1 A from every bead
    wat = w.xyzq[nb:]
    o = _check_waters(wat, w.box)
    oz = np.mod(o[:, 2], 100.0)
    assert np.all((oz >= 70.0 - TOL_POS) | (oz < 30.0 + TOL_POS))
    from scipy.spatial import cKDTree
    tree = cKDTree(np.mod(beads[:, :3], box), boxsize=box)
    sites = np.mod(wat[:, :3].astype(np.float64), box)
    sites = np.where(sites >= box, 0.0, sites)
    d, _ = tree.query(sites, k=1)
    assert d.min() >= 1.0 - TOL_POS
    assert w.xyzq[:, 3].astype(np.float64).sum() == 0.0


def test_serving_stream():
    n_min, n_max = 2000, 9000
    systems = list(W.serving_stream(3, 60, n_min=n_min, n_max=n_max))
    ns = np.array([x.shape[0] for (_, _, _, x) in systems])
    assert np.all(ns % 3 == 0) and np.all((ns >= n_min - 3) & (ns <= n_max + 3))
    # log-uniform sizes: the logs spread evenly over the range (Kolmogorov-Smirnov against uniform)
    from scipy.stats import kstest
    u = (np.log(ns) - math.log(n_min)) / (math.log(n_max) - math.log(n_min))
    assert kstest(u, "uniform").pvalue > 1e-3
    for box, grid, r_c, x in systems[:12]:
        L = box[0]
        assert box == (L, L, L) and r_c == 9.0
        assert abs(x.shape[0] / L ** 3 - 0.1) < 1e-9               # 0.1 charges per A^3
        assert grid[0] % 8 == 0 and grid == (grid[0],) * 3 and abs(grid[0] - L) <= 4.0 + 1e-9
        _check_waters(x, box)
