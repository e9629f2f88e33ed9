"""Pins of the oracle's univariate spline layer against closed forms and identities that do
not come from the oracle itself (Sec. 2 spline spaces S_{p,h}, Sec. 3 embedding P_l)."""
import math

import numpy as np
import pytest

from oracle import bspline


def cardinal_bspline(order, x, deriv=0):
    """Closed form of the cardinal B-spline of the given order (degree order-1) on
    [0, order]: N(x) = 1/(order-1)! sum_j (-1)^j C(order, j) (x-j)_+^(order-1), and its
    derivatives by differentiating the truncated powers."""
    x = np.asarray(x, dtype=float)
    x = np.minimum(x, order - x)     # symmetry about order/2 (even derivatives only)
    assert deriv % 2 == 0
    out = np.zeros_like(x)
    e = order - 1 - deriv
    for j in range(order + 1):
        coef = (-1) ** j * math.comb(order, j) / math.factorial(order - 1)
        coef *= math.factorial(order - 1) / math.factorial(e)  # d^deriv of x^(order-1)
        out += coef * np.where(x - j > 0, (x - j), 0.0) ** e * (x - j > 0)
    return out


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("m", [1, 3, 8])
def test_partition_of_unity_and_nonnegativity(p, m):
    t = bspline.uniform_knots(m, p)
    x = np.concatenate([np.random.default_rng(p * 10 + m).uniform(0, 1, 200), [0.0, 1.0]])
    B = bspline.basis(t, p, x)
    assert B.shape == (len(x), m + p)
    assert np.all(B >= -1e-15)
    np.testing.assert_allclose(B.sum(axis=1), 1.0, atol=1e-14)
    np.testing.assert_allclose(bspline.basis(t, p, x, 1).sum(axis=1), 0.0, atol=1e-10 * m)


def test_hat_functions_p1():
    m = 4
    t = bspline.uniform_knots(m, 1)
    x = np.linspace(0, 1, 41)
    B = bspline.basis(t, 1, x)
    for i in range(m + 1):
        np.testing.assert_allclose(B[:, i], np.maximum(0, 1 - np.abs(x * m - i)), atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6])
def test_integral_closed_form(p):
    m = 7
    t = bspline.uniform_knots(m, p)
    M, _ = bspline.mass_stiffness_1d(t, p)
    # sum_j B_j = 1  =>  (M 1)_i = int B_i = (t_{i+p+1} - t_i) / (p+1)
    expect = np.array([(t[i + p + 1] - t[i]) / (p + 1) for i in range(m + p)])
    np.testing.assert_allclose(M.sum(axis=1), expect, atol=1e-15)
    assert abs(M.sum() - 1.0) < 1e-14


@pytest.mark.parametrize("nq", [1, 2, 3, 5, 7])
def test_gauss_exactness(nq):
    x, w = bspline.gauss_legendre(nq)
    for deg in range(2 * nq):
        assert abs(np.sum(w * x ** deg) - 1.0 / (deg + 1)) < 1e-14
    assert abs(np.sum(w * x ** (2 * nq)) - 1.0 / (2 * nq + 1)) > 1e-12   # not exact beyond 2nq-1


def test_mass_stiffness_p2_rows():
    m = 10
    h = 1.0 / m
    M, K = bspline.mass_stiffness_1d(bspline.uniform_knots(m, 2), 2)
    i = 5
    np.testing.assert_allclose(M[i, i - 2:i + 3], h * np.array([1, 26, 66, 26, 1]) / 120, atol=1e-15)
    np.testing.assert_allclose(K[i, i - 2:i + 3], np.array([-1 / 6, -1 / 3, 1, -1 / 3, -1 / 6]) / h,
                               atol=1e-12)


@pytest.mark.parametrize("p", [2, 3, 4, 5, 6])
def test_interior_rows_are_cardinal_autocorrelations(p):
    m = 4 * p + 4
    h = 1.0 / m
    M, K = bspline.mass_stiffness_1d(bspline.uniform_knots(m, p), p)
    i = m // 2
    ks = np.arange(-p, p + 1)
    order = 2 * p + 2  # autocorrelation of two degree-p cardinal splines: degree 2p+1
    Mrow = h * cardinal_bspline(order, p + 1 + ks)
    Krow = -cardinal_bspline(order, p + 1 + ks, deriv=2) / h
    np.testing.assert_allclose(M[i, i - p:i + p + 1], Mrow, rtol=0, atol=1e-12 * Mrow.max())
    np.testing.assert_allclose(K[i, i - p:i + p + 1], Krow, rtol=0, atol=1e-10 * Krow.max())
    np.testing.assert_allclose(K.sum(axis=1), 0.0, atol=1e-9 * m)
    assert np.all(np.linalg.eigvalsh(M) > 0)
    assert np.all(np.linalg.eigvalsh(K) > -1e-9)


@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_derivatives_reproduce_monomials(p):
    """Splines of degree p contain every polynomial of degree <= p; the coefficients of
    x^a (least squares at many points, exact) must give the analytic derivatives of all
    orders, including one-sided values at 0 and 1."""
    m = 5
    t = bspline.uniform_knots(m, p)
    xs = np.linspace(0, 1, 97)
    B = bspline.basis(t, p, xs)
    xe = np.array([0.0, 0.37, 0.5, 1.0])
    for a in range(p + 1):
        c = np.linalg.lstsq(B, xs ** a, rcond=None)[0]
        for r in range(p + 1):
            got = bspline.basis(t, p, xe, r) @ c
            coef = math.factorial(a) / math.factorial(a - r) if r <= a else 0.0
            expect = coef * xe ** (a - r) if r <= a else np.zeros_like(xe)
            np.testing.assert_allclose(got, expect, atol=1e-9 * m ** r)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6])
@pytest.mark.parametrize("mc", [1, 2, 5])
def test_knot_insertion_reproduces_coarse_splines(p, mc):
    P = bspline.prolongation_1d(mc, p)
    assert P.shape == (2 * mc + p, mc + p)
    np.testing.assert_allclose(P.sum(axis=1), 1.0, atol=1e-14)
    c = np.random.default_rng(p + 7 * mc).normal(size=mc + p)
    x = np.random.default_rng(1).uniform(0, 1, 300)
    coarse = bspline.basis(bspline.uniform_knots(mc, p), p, x) @ c
    fine = bspline.basis(bspline.uniform_knots(2 * mc, p), p, x) @ (P @ c)
    np.testing.assert_allclose(fine, coarse, atol=1e-14)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_knot_insertion_interior_stencil_lane_riesenfeld(p):
    mc = 3 * p + 6
    P = bspline.prolongation_1d(mc, p)
    j = mc // 2 + p // 2
    col = P[:, j]
    nz = np.nonzero(np.abs(col) > 1e-15)[0]
    stencil = np.array([math.comb(p + 1, i) for i in range(p + 2)]) / 2 ** p
    np.testing.assert_allclose(col[nz[0]:nz[0] + p + 2], stencil, atol=1e-15)
    assert len(nz) == p + 2
