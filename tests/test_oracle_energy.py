"""Pins of the oracle's energies, potentials and forces against closed forms and
independent methods (no GPU): the NaCl Madelung constant, classic Ewald sums,
a real-space image sum of the far Gaussians, Eq. 33's truncation bound,
finite differences and exact invariances."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import series as S
from paper_1911_01377_gb300 import workloads as W

MADELUNG_NACL = 1.7475645946331822   # rock-salt Madelung constant (nearest-neighbour distance 1)


def _ser(tables, key):
    return O.Series(*tables[key])


def _nacl(m):
    """Rock salt, m^3 conventional cells of edge 2 (nearest-neighbour distance 1)."""
    rows = []
    for i in range(2 * m):
        for j in range(2 * m):
            for k in range(2 * m):
                rows.append((i, j, k, 1.0 if (i + j + k) % 2 == 0 else -1.0))
    a = np.array(rows, dtype=np.float64)
    return a[:, :3], a[:, 3], (2.0 * m,) * 3


def test_madelung_nacl(tables):
    pos, q, box = _nacl(2)
    pairs = q.size / 2
    # classic Ewald, the independent route to the same constant
    E, phi, f = O.ewald(box, pos, q)
    assert abs(E / pairs + MADELUNG_NACL) < 1e-13
    assert np.max(np.abs(f)) < 1e-12
    # most accurate u-series of Table 1 (M_b = 3.9e-11)
    r = O.evaluate(_ser(tables, "table1_c"), box[0] / 2, box, pos, q)
    assert abs(r.E / pairs / -MADELUNG_NACL - 1.0) < 1e-8
    assert np.max(np.abs(r.F)) < 1e-10
    # phi_i = dE/dq_i: every ion sees -/+ M
    assert np.max(np.abs(r.phi * q + MADELUNG_NACL)) < 2e-8
    # recommended b = 2 C1 (M_b = 2.3e-3): deviation of the order of M_b
    r2 = O.evaluate(_ser(tables, "table2_C1"), box[0] / 2, box, pos, q)
    dev = abs(r2.E / pairs / -MADELUNG_NACL - 1.0)
    assert 1e-5 < dev < 3 * S.M_b(2.0)


@pytest.mark.parametrize("seed", [1, 2])
def test_against_classic_ewald(tables, seed):
    box = (9.0, 10.0, 11.0)
    xyzq = W.random_neutral(seed, 48, box, min_dist=1.2)
    pos, q = xyzq[:, :3], xyzq[:, 3]
    E, phi, f = O.ewald(box, pos, q)
    r = O.evaluate(_ser(tables, "table1_c"), 4.4, box, pos, q)
    assert abs(r.E / E - 1.0) < 1e-9
    assert O.rms_rel(r.F, f) < 1e-9
    assert O.rms_rel(r.phi, phi) < 1e-9
    # b = 2: errors of the order of M_b
    r2 = O.evaluate(_ser(tables, "table2_C1"), 4.4, box, pos, q)
    assert abs(r2.E / E - 1.0) < 3 * S.M_b(2.0)
    assert O.rms_rel(r2.F, f) < 10 * S.M_b(2.0)


@pytest.mark.parametrize("key,n_terms", [("table2_C1", 3), ("table2_C2", 4), ("table1_a", 5)])
def test_far_kspace_equals_realspace_image_sum(tables, key, n_terms):
    # Poisson summation: the k-space far sum with the first N Gaussians equals
    # their periodic real-space image sum (neutral system, k = 0 term absent).
    box = (7.0, 8.0, 9.0)
    xyzq = W.random_neutral(5, 24, box, min_dist=1.0)
    pos, q = xyzq[:, :3], xyzq[:, 3]
    assert float(np.sum(q.astype(np.float64))) == 0.0
    ser = _ser(tables, key)
    r_c = 3.2
    Ek, pk, fk, _ = O.far(ser, r_c, box, pos, q, n_terms=n_terms)
    Er, pr, fr = O.far_realspace(ser, r_c, box, pos, q, n_terms=n_terms)
    assert abs(Ek / Er - 1.0) < 1e-11
    assert O.rms_rel(pk, pr) < 1e-11
    assert O.rms_rel(fk, fr) < 1e-10


def test_truncation_bound_eq33(tables):
    # App. F: the relative error of the far energy truncated to N terms is
    # below exp(2 N ln b - 2 (b^{2N} - 1) pi^2 sigma^2 / L^2), L = max side.
    box = (16.0, 18.0, 22.0)
    xyzq = W.random_neutral(7, 96, box, min_dist=1.0)
    pos, q = xyzq[:, :3], xyzq[:, 3]
    ser = _ser(tables, "table2_C1")
    r_c = 6.0
    sigma = r_c / ser.r0
    Einf, _, _, _ = O.far(ser, r_c, box, pos, q)
    seen_tight = False
    for N in range(1, 7):
        EN, _, _, _ = O.far(ser, r_c, box, pos, q, n_terms=N)
        rel = abs(EN - Einf) / abs(Einf)
        bound = S.trunc_bound(N, ser.b, sigma, max(box))
        assert rel <= bound * (1 + 1e-9) + 1e-15
        assert EN <= Einf * (1 + 1e-15)               # every dropped term is positive
        if 1e-12 < bound < 1:
            seen_tight = True
    assert seen_tight


def test_quadratic_form_and_invariances(tables):
    box = (12.0, 12.5, 13.0)
    xyzq = W.random_neutral(11, 64, box, min_dist=1.0)
    pos, q = xyzq[:, :3].astype(np.float64), xyzq[:, 3].astype(np.float64)
    ser = _ser(tables, "table2_C1")
    r_c = 5.0
    r = O.evaluate(ser, r_c, box, pos, q)
    # E = 1/2 sum q_i phi_i (E is a quadratic form, phi = dE/dq)
    assert abs(0.5 * np.dot(q, r.phi) / r.E - 1.0) < 1e-12
    # no net force
    assert np.max(np.abs(r.F.sum(axis=0))) < 1e-11 * np.max(np.abs(r.F))
    # translation invariance
    shift = np.array([3.3, -1.7, 25.2])
    rt = O.evaluate(ser, r_c, box, pos + shift, q)
    assert abs(rt.E / r.E - 1.0) < 1e-12
    assert O.rms_rel(rt.F, r.F) < 1e-11
    # Eq. 23 scaling: E(lambda x, lambda L, lambda r_c) = E / lambda
    lam = 1.7
    rs = O.evaluate(ser, lam * r_c, tuple(lam * np.array(box)), lam * pos, q)
    assert abs(rs.E * lam / r.E - 1.0) < 1e-12
    assert O.rms_rel(rs.F * lam * lam, r.F) < 1e-11
    # energy breakdown adds up and the self term is -F(0)/2 sum q^2
    assert abs(r.E_near + r.E_far + r.E_self - r.E) < 1e-12 * abs(r.E)
    assert abs(r.E_self + 0.5 * O.F0(ser, r_c) * np.dot(q, q)) < 1e-12 * abs(r.E_self)


def test_finite_differences(tables):
    box = (11.0, 12.0, 13.0)
    xyzq = W.random_neutral(13, 40, box, min_dist=1.0)
    pos, q = xyzq[:, :3].astype(np.float64), xyzq[:, 3].astype(np.float64)
    ser = _ser(tables, "table2_C1")
    r_c = 5.0
    r = O.evaluate(ser, r_c, box, pos, q)
    h = 1e-4
    for i in (0, 7, 23):
        for a in range(3):
            p1 = pos.copy(); p1[i, a] += h
            p2 = pos.copy(); p2[i, a] -= h
            fd = -(O.evaluate(ser, r_c, box, p1, q).E - O.evaluate(ser, r_c, box, p2, q).E) / (2 * h)
            assert abs(fd - r.F[i, a]) < 1e-7 * max(1.0, abs(r.F[i, a]))
        q1 = q.copy(); q1[i] += h
        q2 = q.copy(); q2[i] -= h
        fdq = (O.evaluate(ser, r_c, box, pos, q1).E - O.evaluate(ser, r_c, box, pos, q2).E) / (2 * h)
        assert abs(fdq - r.phi[i]) < 1e-8 * max(1.0, abs(r.phi[i]))


def test_pair_energy_continuous_across_rc(tables):
    # a +1/-1 pair in a large box: E(d) is continuous across r_c, and for the C1
    # construction so is dE/dd (Eqs. 20-26)
    box = (40.0, 40.0, 40.0)
    r_c = 6.0
    for key, smooth in (("table2_C0", 0), ("table2_C1", 1)):
        ser = _ser(tables, key)
        q = np.array([1.0, -1.0])

        def E(d):
            pos = np.array([[10.0, 10.0, 10.0], [10.0 + d, 10.0, 10.0]])
            return O.evaluate(ser, r_c, box, pos, q).E

        eps = 1e-10
        left, right = E(r_c - eps), E(r_c + eps)
        assert abs(left - right) < 1e-10          # slope ~ 1/r_c^2 contributes ~1e-11
        if smooth:
            h = 1e-4
            sl = (E(r_c - eps) - E(r_c - eps - h)) / h
            sr = (E(r_c + eps + h) - E(r_c + eps)) / h
            assert abs(sl - sr) < 1e-5                # one-sided slopes agree to O(h)


def test_canonical_pairs_match_exact_distances(tables):
    # the single-precision pair predicate lists exactly the pairs closer than
    # r_c (in double precision on the same inputs), up to pairs within a
    # rounding of the cutoff
    w = W.get("water_3k")
    box, r_c = w.box, w.r_c[0]
    nc = [int(math.floor(L / r_c)) for L in box]
    cnt, h = O.canon_pairs(w.xyzq, box, nc, r_c)
    pos = w.xyzq[:, :3].astype(np.float64)
    d = pos[:, None, :] - pos[None, :, :]
    d -= np.array(box) * np.round(d / np.array(box))
    r2 = np.sum(d * d, axis=-1)
    np.fill_diagonal(r2, np.inf)
    exact = (r2 < r_c * r_c).sum(axis=1)
    border = (np.abs(np.sqrt(r2) - r_c) < 1e-4).sum(axis=1)
    assert np.all(np.abs(cnt - exact) <= border)
    assert cnt.sum() % 2 == 0
    # cells: every wrapped coordinate lies in its cell and in [0, L)
    cell, xw = O.canon_cells(w.xyzq, box, nc)
    assert np.all(xw >= 0) and np.all(xw < np.array(box, dtype=np.float32))
    cz, rem = np.divmod(cell, nc[0] * nc[1])
    cy, cx = np.divmod(rem, nc[0])
    for a, c in enumerate((cx, cy, cz)):
        width = box[a] / nc[a]
        assert np.all(xw[:, a] >= c * width - 1e-4) and np.all(xw[:, a] < (c + 1) * width + 1e-4)


def test_virial_kspace_equals_realspace(tables):
    # Poisson summation for the strain derivative: the k-space far virial of the
    # first N Gaussians equals their real-space pair virial (neutral system)
    box = (7.0, 8.0, 9.0)
    xyzq = W.random_neutral(5, 24, box, min_dist=1.0)
    pos, q = xyzq[:, :3], xyzq[:, 3]
    ser = _ser(tables, "table2_C1")
    r_c = 3.2
    _, wk = O.virial(ser, r_c, box, pos, q, n_terms=3)
    wr = O.far_virial_realspace(ser, r_c, box, pos, q, n_terms=3)
    assert np.max(np.abs(wk - wr)) < 1e-10 * np.max(np.abs(wr))
    assert np.allclose(wk, wk.T, rtol=0, atol=1e-14 * np.max(np.abs(wk)))


def test_virial_diagonal_is_strain_derivative(tables):
    # W_aa = -dE/d(eps_aa): stretch axis a of the box and every position by
    # (1 +- h) and difference the full energy (near + far + self)
    box = np.array([10.0, 11.0, 12.0])
    xyzq = W.random_neutral(17, 40, tuple(box), min_dist=1.0)
    pos, q = xyzq[:, :3].astype(np.float64), xyzq[:, 3].astype(np.float64)
    ser = _ser(tables, "table2_C1")
    r_c = 4.5
    wn, wf = O.virial(ser, r_c, box, pos, q)
    Wt = wn + wf
    h = 1e-5
    for a in range(3):
        s = np.ones(3)
        s[a] = 1 + h
        Ep = O.evaluate(ser, r_c, tuple(box * s), pos * s, q).E
        s[a] = 1 - h
        Em = O.evaluate(ser, r_c, tuple(box * s), pos * s, q).E
        fd = -(Ep - Em) / (2 * h)
        assert abs(fd - Wt[a, a]) < 1e-6 * max(1.0, abs(Wt[a, a]))
    # near part alone is the pair sum 1/2 sum d (x) f: its trace equals sum_i r_i . F_i^near
    # only without images; here just check symmetry
    assert np.allclose(wn, wn.T, rtol=0, atol=1e-13 * np.max(np.abs(wn)))


def test_virial_off_diagonal_near_is_shear_derivative(tables):
    # Off-diagonal components of the near virial, pinned by a shear.  The charges
    # form a cluster of radius 4 A in a 40 A box with r_c = 5.5 A, so no pair
    # inside r_c crosses the periodic boundary and E_near is a plain pair sum of
    # Eq. 20.  Shearing the positions alone (x_a += eps x_b, box unchanged) gives
    # dE_near/d eps = -sum_i F_i,a x_i,b = -W_near,ab, the pair-virial component
    # a, b (the centre of the cluster drops out because the near forces sum to
    # zero).  A swapped or misplaced off-diagonal slot in the oracle's near
    # virial fails this for some (a, b).
    rng = np.random.default_rng(23)
    box = np.array([40.0, 40.0, 40.0])
    centre = box / 2
    pts = []
    while len(pts) < 30:
        p = centre + rng.uniform(-4.0, 4.0, 3)
        if np.linalg.norm(p - centre) < 4.0 and all(np.linalg.norm(p - o) >= 1.0 for o in pts):
            pts.append(p)
    pos = np.array(pts)
    q = rng.normal(0.0, 0.6, len(pts))
    q -= q.mean()
    ser = _ser(tables, "table2_C1")
    r_c = 5.5
    wn, _ = O.virial(ser, r_c, box, pos, q)
    assert np.max(np.abs(wn - np.diag(np.diag(wn)))) > 1e-3   # the off-diagonal part is not trivially zero
    h = 1e-6
    for a, b in [(0, 1), (1, 0), (0, 2), (2, 0), (1, 2), (2, 1)]:
        def e_near(eps):
            p = pos.copy()
            p[:, a] += eps * (pos[:, b] - centre[b])
            return O.evaluate(ser, r_c, tuple(box), p, q).E_near
        fd = -(e_near(h) - e_near(-h)) / (2 * h)
        assert abs(fd - wn[a, b]) < 1e-7 * max(1.0, np.max(np.abs(wn))), (a, b, fd, wn[a, b])
