"""The two-level form of a wide Gaussian term (the multilevel remark at the end of Sec. V), checked in 1D on the
CPU against the plain definition.

Per axis a term's deconvolved kernel e_w(x) = exp(-x^2 / 2w^2) is the convolution of three Gaussians of widths
a, c, b with a^2 + b^2 + c^2 = w^2:  e_w = w / (2 pi a b c) (e_b * e_c * e_a).  With the two outer integrals taken
as sums over a grid of spacing H = 2h, applying e_w to a fine-grid function becomes restriction (e_a, onto the
coarse points), the ordinary coarse pass (e_c) and prolongation (e_b), with the factor H^2 w / (2 pi a b c).
This test writes that chain out with numpy for a delta function and compares it with e_w sampled on the fine
grid, for the widths the plan sends to the coarse grid (at least 2.25 H) and the transfer width a = b = 1.3 H
the library uses, with the 33-tap truncation of the transfers.  The sums replace the integrals with an error of
about exp(-2 pi^2 v^2 / H^2), v the narrowest width in the integrand: far below the 1e-6 asserted here.
"""
import math

import numpy as np
import pytest


def periodic_gauss(x, s, period):
    """exp(-x^2 / 2 s^2) summed over the periodic images."""
    return sum(np.exp(-(x + m * period) ** 2 / (2.0 * s * s)) for m in range(-3, 4))


@pytest.mark.parametrize("n,h", [(96, 1.04), (176, 1.25), (64, 1.25)])
@pytest.mark.parametrize("w_over_H", [2.25, 3.0, 5.0, 9.0])
def test_two_level_factorisation_reproduces_the_fine_kernel(n, h, w_over_H):
    H = 2.0 * h
    L = n * h
    w = w_over_H * H
    a = b = 1.3 * H
    c = math.sqrt(w * w - a * a - b * b)
    T = 16                                            # transfer half-width in fine points (6 a / h = 15.6)
    g = np.arange(n) * h                              # fine points
    G = np.arange(n // 2) * H                         # coarse points (fine index 2 G)
    # restriction of a delta at fine point 0: r(G) = e_a(2G h - 0), taps |2G - 0| <= T (periodic)
    t_idx = np.arange(-T, T + 1)
    r = np.zeros(n // 2)
    for t in t_idx:                                   # fine point 0 feeds coarse G with 2G = -t (mod n)
        if t % 2 == 0:
            r[(-t // 2) % (n // 2)] += periodic_gauss(t * h, a, L)
    # coarse pass with the periodised e_c
    Cmat = periodic_gauss(G[:, None] - G[None, :], c, L)
    tc = Cmat @ r
    # prolongation: f(g) = sum over coarse G with |g - 2G| <= T of e_b(g - 2G)
    out = np.zeros(n)
    for gi in range(n):
        for Gi in range(n // 2):
            d = gi - 2 * Gi
            d = (d + n // 2) % n - n // 2             # nearest periodic offset in fine points
            if abs(d) <= T:
                out[gi] += periodic_gauss(d * h, b, L) * tc[Gi]
    out *= H * H * w / (2.0 * math.pi * a * b * c)
    ref = periodic_gauss(g, w, L)                     # the fine pass applied to the same delta: e_w(g h)
    err = np.max(np.abs(out - ref)) / np.max(np.abs(ref))
    assert err < 1e-6, err


def test_threshold_keeps_the_coarse_kernel_resolved():
    """With a = b = 1.3 H, a width w >= 2.25 H leaves c = sqrt(w^2 - 2 a^2) >= 1.3 H, so the coarse kernel is as
    well resolved on the coarse grid as the transfers are on the fine one."""
    H = 1.0
    a = 1.3 * H
    c = math.sqrt((2.25 * H) ** 2 - 2 * a * a)
    assert c >= 1.29 * H
    # the grid-sum error bound exp(-2 pi^2 v^2 / H^2) at the narrowest width v = 1.3 H
    assert math.exp(-2 * math.pi ** 2 * 1.3 ** 2) < 1e-14
