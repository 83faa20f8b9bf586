"""Series construction in plain FP64 (numpy): the defining equations of the
u-series parameters, written out for the tests.  Test infrastructure only.

F^1(r) denotes the far part at sigma = 1:
    F^1(r) = 2 ln(b) [ w0 G_1(r / s0) + sum_{j>=1} b^-j G_1(b^-j r) ]     Eqs. 24, 28
with G_1(r) = exp(-r^2 / 2) / sqrt(2 pi) (Sec. III.A; for the C2 construction
the narrow term is read unnormalised in s0, see the Eq. 28 note in the oracle).

    C0: r0 = smallest root of r F^1(r) - 1 with w0 = 1           (Eqs. 19, 21)
    C1: F^1(r0) = 1/r0 and F^1'(r0) = -1/r0^2                     (Eqs. 25, 26)
    C2 point of the C1 family: also F^1''(r0) = 2/r0^3            (Eq. 27)
    M_b = 2^{3/2} exp(-pi^2 / (2 ln b))                           (Eq. 14)
    M(alpha, b), the 1/r^alpha generalisation                     (Eq. B3)
    truncation bound exp(2 N ln b - 2 (b^{2N} - 1) pi^2 sigma^2 / L^2)   (Eq. 33)
"""
from __future__ import annotations

import math

import numpy as np

_SQ2PI = math.sqrt(2.0 * math.pi)


def _nterms(b: float) -> int:
    return int(math.ceil(50.0 * math.log(10.0) / math.log(b))) + 2


def far1(r, b, w0=1.0, s0=1.0, deriv: int = 0):
    """d^deriv/dr^deriv F^1(r) (deriv = 0, 1, 2), sigma = 1."""
    r = np.asarray(r, dtype=np.float64)
    lb = math.log(b)
    out = np.zeros_like(r)
    # term j = 0: w0 exp(-r^2 / (2 s0^2)) / sqrt(2 pi)
    terms = [(w0, s0)] + [(b ** -j, b ** j) for j in range(1, _nterms(b))]
    for amp, s in terms:
        g = amp * np.exp(-r * r / (2.0 * s * s)) / _SQ2PI
        if deriv == 0:
            out += g
        elif deriv == 1:
            out += g * (-r / (s * s))
        elif deriv == 2:
            out += g * (r * r / s ** 4 - 1.0 / (s * s))
    return 2.0 * lb * out


def bsa(r, b, sigma=1.0):
    """Bilateral series approximation B_b^sigma(r) of Eq. 11."""
    r = np.asarray(r, dtype=np.float64)
    lb = math.log(b)
    J = _nterms(b)
    out = np.zeros_like(r)
    for j in range(-J, J + 1):
        bj = b ** (-j)
        out += bj * np.exp(-0.5 * (bj * r / sigma) ** 2)
    return 2.0 * lb * out / (_SQ2PI * sigma)


def M_b(b: float) -> float:
    """Asymptotic relative-error bound of Eq. 14."""
    return 2.0 ** 1.5 * math.exp(-math.pi ** 2 / (2.0 * math.log(b)))


def M_alpha(alpha: float, b: float) -> float:
    """Asymptotic relative-error bound of the BSA of 1/r^alpha, Eq. B3."""
    d = math.log(b)
    return (2.0 * math.sqrt(2.0 * math.pi) / math.gamma(alpha / 2.0)
            * (alpha * alpha / 4.0 + math.pi ** 2 / d ** 2) ** ((alpha - 1.0) / 4.0)
            * math.exp(-math.pi ** 2 / (2.0 * d)))


def trunc_bound(N: int, b: float, sigma: float, L: float) -> float:
    """Relative truncation bound of Eq. 33 / Eq. F4 for N terms."""
    return math.exp(2.0 * N * math.log(b) - 2.0 * (b ** (2 * N) - 1.0) * math.pi ** 2 * sigma ** 2 / L ** 2)


def solve_c0(b: float, r_guess: float, iters: int = 60) -> float:
    """Root of r F^1(r) - 1 (Eq. 21) by Newton's method from r_guess."""
    r = r_guess
    for _ in range(iters):
        f = r * far1(r, b) - 1.0
        df = far1(r, b) + r * far1(r, b, deriv=1)
        step = f / df
        r -= step
        if abs(step) < 1e-16 * r:
            break
    return float(r)


def w0_of_r0(r0: float, b: float) -> float:
    """Eq. 25: the w0 that makes F^1(r0) = 1/r0 (C1 construction, s0 = 1)."""
    lb = math.log(b)
    tail = sum(b ** -j * math.exp(-0.5 * (r0 / b ** j) ** 2) / _SQ2PI for j in range(1, _nterms(b)))
    g1 = math.exp(-0.5 * r0 * r0) / _SQ2PI
    return (1.0 / (2.0 * lb * r0) - tail) / g1


def solve_c1(b: float, r_guess: float, iters: int = 80):
    """Eq. 26 with w0 from Eq. 25: returns (r0, w0)."""
    def h(r):
        w = w0_of_r0(r, b)
        return float(far1(r, b, w0=w, deriv=1)) + 1.0 / (r * r)

    r = r_guess
    for _ in range(iters):
        e = 1e-7 * r
        d = (h(r + e) - h(r - e)) / (2.0 * e)
        step = h(r) / d
        r -= step
        if abs(step) < 1e-15 * r:
            break
    return float(r), w0_of_r0(r, b)


def c2_residuals(b: float, r0: float, w0: float, s0: float = 1.0):
    """Residuals of the three conditions of Eq. 27 (scaled by r0, r0^2, r0^3)."""
    f0 = float(far1(r0, b, w0, s0))
    f1 = float(far1(r0, b, w0, s0, deriv=1))
    f2 = float(far1(r0, b, w0, s0, deriv=2))
    return np.array([r0 * f0 - 1.0, r0 * r0 * f1 + 1.0, r0 ** 3 * f2 - 2.0])


def solve_c2(b: float, r0: float, w0: float, iters: int = 40):
    """Newton's method on Eq. 27 in the unknowns (b, r0, w0), s0 = 1."""
    x = np.array([b, r0, w0], dtype=np.float64)
    for _ in range(iters):
        F = c2_residuals(*x)
        J = np.zeros((3, 3))
        for k in range(3):
            e = np.zeros(3)
            e[k] = 1e-7 * abs(x[k])
            J[:, k] = (c2_residuals(*(x + e)) - c2_residuals(*(x - e))) / (2.0 * e[k])
        step = np.linalg.solve(J, F)
        x = x - step
        if np.max(np.abs(step) / np.abs(x)) < 1e-15:
            break
    return tuple(float(v) for v in x)
