"""Pins of the oracle's lattice fundamental solution against what the paper fixes.

phi is defined by the Fourier integral eq. 1.8; A phi = delta follows from it and
eq. 1.2.  The oracle builds phi by an exact rational recursion; these tests tie
that table to the definition (2-D quadrature of eq. 1.8), to Remark 3.1's
one-dimensional form, to closed forms, and to the asymptotic expansion eq. 3.1.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy import integrate

import oracle
from oracle.phi_exact import octant_index, phi_exact_fraction, phi_octant

PI = math.pi
EULER_GAMMA = 0.5772156649015329


def exact(m1, m2):
    """Correctly rounded phi(m1, m2) from the exact octant (a + b/pi evaluated exactly)."""
    hi, lo = max(abs(m1), abs(m2)), min(abs(m1), abs(m2))
    return float(phi_octant(128)[octant_index(hi, lo)])


def test_closed_forms_exact():
    # phi(0) = 0 (eq. 1.8), phi(e1) - phi(0) = -1/4, phi(1,1) - phi(0) = -1/pi
    assert phi_exact_fraction(0, 0, R=4) == (Fraction(0), Fraction(0))
    assert phi_exact_fraction(1, 0, R=4) == (Fraction(-1, 4), Fraction(0))
    assert phi_exact_fraction(0, -1, R=4) == (Fraction(-1, 4), Fraction(0))
    assert phi_exact_fraction(1, 1, R=4) == (Fraction(0), Fraction(-1))
    # derived: phi(2,0) = -1 + 2/pi, phi(2,1) = 1/4 - 2/pi, phi(2,2) = -4/(3 pi)
    assert phi_exact_fraction(2, 0, R=4) == (Fraction(-1), Fraction(2))
    assert phi_exact_fraction(2, 1, R=4) == (Fraction(1, 4), Fraction(-2))
    assert phi_exact_fraction(2, 2, R=4) == (Fraction(0), Fraction(-4, 3))


def test_table_independent_of_radius():
    small = phi_octant(40)
    big = phi_octant(128)
    assert np.array_equal(small, big[: small.size])


@pytest.mark.parametrize("m", [(1, 0), (1, 1), (2, 1), (3, 0), (3, 2), (4, 4), (5, 1), (6, 3), (8, 0)])
def test_definition_eq_1_8_by_2d_quadrature(m):
    """eq. 1.8 integrated directly (cos(t1 m1) cos(t2 m2) part; the odd part vanishes)."""
    m1, m2 = m

    def integrand(t2, t1):
        den = 4.0 * math.sin(t1 / 2) ** 2 + 4.0 * math.sin(t2 / 2) ** 2
        if den == 0.0:
            return 0.0
        return (math.cos(m1 * t1) * math.cos(m2 * t2) - 1.0) / den

    val, err = integrate.dblquad(integrand, 0, PI, 0, PI, epsabs=1e-13, epsrel=1e-13)
    assert abs(val / PI ** 2 - exact(m1, m2)) < 1e-13


@pytest.mark.parametrize("m", [(0, 7), (3, 11), (12, 5), (20, 0), (17, 17), (31, 9), (40, 2)])
def test_remark_3_1_one_dimensional_form(m):
    """Remark 3.1: integrate t1 in closed form, leaving
    phi(m) = (1/pi) int_0^pi (exp(-|m1| s) cos(m2 t) - 1) / (2 sinh s) dt,  cosh s = 2 - cos t.
    (cosh s = 1 + 2 sin^2(t/2) gives s = 2 asinh(sin(t/2)), sinh s = 2 sin(t/2) sqrt(1 + sin^2(t/2)).)"""
    m1, m2 = m

    # composite 40-point Gauss-Legendre on 64 panels (nodes avoid t = 0)
    x, w = np.polynomial.legendre.leggauss(40)
    edges = np.linspace(0.0, PI, 65)
    t = (0.5 * (edges[1:, None] - edges[:-1, None]) * x[None, :] + 0.5 * (edges[1:, None] + edges[:-1, None])).ravel()
    wt = (0.5 * (edges[1:, None] - edges[:-1, None]) * w[None, :]).ravel()
    h = np.sin(t / 2)
    s = 2.0 * np.arcsinh(h)
    num = np.expm1(-abs(m1) * s) * np.cos(m2 * t) - 2.0 * np.sin(m2 * t / 2) ** 2
    val = math.fsum(wt * num / (4.0 * h * np.sqrt(1.0 + h * h)))
    assert abs(val / PI - exact(m1, m2)) < 5e-15


def test_A_phi_is_delta_on_table():
    R = 64
    oct_ = phi_octant(R)

    def p(x, y):
        x, y = abs(x), abs(y)
        hi, lo = max(x, y), min(x, y)
        return oct_[octant_index(hi, lo)]

    for x in range(-R + 1, R):
        for y in range(-R + 1, R):
            a = 4 * p(x, y) - p(x + 1, y) - p(x - 1, y) - p(x, y + 1) - p(x, y - 1)
            assert abs(a - (1.0 if (x, y) == (0, 0) else 0.0)) < 1e-9 * (1 + abs(x) + abs(y)), (x, y)


def test_symmetry_d4():
    d = np.array([(3, 7), (-3, 7), (3, -7), (-3, -7), (7, 3), (-7, 3), (7, -3), (-7, -3)])
    v = oracle.phi(d)
    assert np.all(v == v[0])
    d2 = np.array([(300, 77), (-77, 300), (77, -300), (-300, -77)])  # asymptotic branch
    v2 = oracle.phi(d2)
    assert np.allclose(v2, v2[0], rtol=0, atol=1e-15)


def test_asymptotic_eq_3_1_against_exact_table():
    """eq. 3.1 with its O(|m|^-6) remainder dropped tracks the exact table with an
    error that decays like |m|^-6; the paper's '1e-12 for |m| > 30' is optimistic
    (measured ~2.1e-10 at |m| = 30)."""
    R = 256
    oct_ = phi_octant(R)
    pts = [(hi, lo) for hi in range(30, R + 1, 7) for lo in range(0, hi + 1, 5)]
    d = np.array(pts, dtype=np.float64)
    asym = oracle.phi_asym(d)
    ex = np.array([oct_[octant_index(h, l)] for h, l in pts])
    r = np.hypot(d[:, 0], d[:, 1])
    err = np.abs(asym - ex)
    assert np.all(err <= 0.2 / r ** 6 + 4e-16)
    assert err.max() > 1e-11  # the remainder is really there near |m| = 30
    # at the oracle's switch radius the remainder is below binary64 resolution of phi
    far = [(256, 0), (256, 100), (256, 256)]
    e_far = np.abs(oracle.phi_asym(np.array(far, float)) - np.array([oct_[octant_index(*p)] for p in far]))
    assert e_far.max() < 1e-15


def test_log_slope_and_constant():
    """phi(m) + (1/2pi) log|m| -> -(1/2pi)(gamma + log(8)/2) (eq. 3.1 leading term)."""
    oct_ = phi_octant(256)
    c = -(EULER_GAMMA + 0.5 * math.log(8.0)) / (2 * PI)
    for hi, lo in [(200, 0), (256, 256), (256, 31)]:
        v = oct_[octant_index(hi, lo)] + math.log(math.hypot(hi, lo)) / (2 * PI)
        assert abs(v - c) < 1e-5
    # slope along an axis: phi(2m) - phi(m) = -(1/2pi) log 2 + (1/24pi)(1/(2m)^2 - 1/m^2) + O(m^-4)
    v = oct_[octant_index(256, 0)] - oct_[octant_index(128, 0)]
    pred = -math.log(2) / (2 * PI) + (1.0 / 256 ** 2 - 1.0 / 128 ** 2) / (24 * PI)
    assert abs(v - pred) < 1e-10
    assert abs(v + math.log(2) / (2 * PI)) > 1e-7


def test_phi_switches_to_asymptotic_beyond_table():
    R = 64
    inside = oracle.phi(np.array([[64, 10]]), R=R)[0]
    outside = oracle.phi(np.array([[65, 10]]), R=R)[0]
    assert inside == phi_octant(R)[octant_index(64, 10)]
    assert outside == oracle.phi_asym(np.array([[65.0, 10.0]]))[0]
    assert abs(outside - exact(65, 10)) < 0.2 / (65 ** 2 + 100) ** 3
    assert abs(outside - exact(65, 10)) > 1e-14
