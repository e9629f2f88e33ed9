"""Univariate splines S_{p,h}(0,1) of maximum smoothness (Sec. 2), Gauss-Legendre
quadrature, the univariate mass and stiffness matrices M, K used by the edge/face
smoothers (Sec. 3), and the canonical embedding between nested spline spaces (Sec. 3,
the matrix P_l) by Boehm knot insertion.

Everything is FP64 NumPy and follows the textbook definitions: Cox-de Boor recursion for
values and derivatives, Boehm's single-knot insertion applied once per new knot.
"""
from __future__ import annotations

import numpy as np


def uniform_knots(m: int, p: int) -> np.ndarray:
    """Open uniform knot vector on [0,1] with m intervals: p+1 zeros, i/m, p+1 ones.
    Its n = m + p B-splines span S_{p,1/m}(0,1) of Sec. 2 (maximum smoothness C^{p-1})."""
    return np.concatenate([np.zeros(p + 1), np.arange(1, m) / m, np.ones(p + 1)])


def intervals_of(knots: np.ndarray, p: int) -> int:
    """Number of intervals m of an open uniform knot vector; raises if it is not one."""
    t = np.asarray(knots, dtype=np.float64)
    m = len(t) - 2 * p - 1
    if m < 1 or not np.allclose(t, uniform_knots(m, p), atol=1e-14, rtol=0):
        raise ValueError("knot vector is not open uniform on [0,1]")
    return m


def basis(t: np.ndarray, p: int, x, deriv: int = 0) -> np.ndarray:
    """Matrix B[q, i] = d^deriv/dx^deriv B_{i,p}(x_q) by the Cox-de Boor recursion.

    Degree-0 functions are interval indicators (the last non-empty interval is closed on
    the right so that x = 1 is covered).  The value recursion
        B_{i,k} = (x-t_i)/(t_{i+k}-t_i) B_{i,k-1} + (t_{i+k+1}-x)/(t_{i+k+1}-t_{i+1}) B_{i+1,k-1}
    raises the degree to p-deriv, then the derivative recursion
        D B_{i,k} = k/(t_{i+k}-t_i) B_{i,k-1} - k/(t_{i+k+1}-t_{i+1}) B_{i+1,k-1}
    is applied `deriv` times (0/0 := 0 throughout)."""
    t = np.asarray(t, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    nint = len(t) - 1
    B = np.zeros((len(x), nint))
    nonempty = [i for i in range(nint) if t[i] < t[i + 1]]
    for i in nonempty:
        B[:, i] = (t[i] <= x) & (x < t[i + 1])
    B[x == t[-1], nonempty[-1]] = 1.0
    for k in range(1, p + 1):
        newB = np.zeros((len(x), nint - k))
        for i in range(nint - k):
            d1 = t[i + k] - t[i]
            d2 = t[i + k + 1] - t[i + 1]
            if k > p - deriv:
                a = k / d1 if d1 > 0 else 0.0
                b = k / d2 if d2 > 0 else 0.0
                newB[:, i] = a * B[:, i] - b * B[:, i + 1]
            else:
                a = (x - t[i]) / d1 if d1 > 0 else np.zeros_like(x)
                b = (t[i + k + 1] - x) / d2 if d2 > 0 else np.zeros_like(x)
                newB[:, i] = a * B[:, i] + b * B[:, i + 1]
        B = newB
    return B


def gauss_legendre(nq: int):
    """nq-point Gauss-Legendre rule on [0,1] (library routine leggauss, mapped)."""
    xg, wg = np.polynomial.legendre.leggauss(nq)
    return 0.5 * (xg + 1.0), 0.5 * wg


def quadrature_points(t: np.ndarray, p: int, nq: int | None = None):
    """Element-wise Gauss rule with nq = p+1 points per non-empty knot interval:
    returns (x, w, elem) where elem[q] is the interval index of point q."""
    nq = p + 1 if nq is None else nq
    xr, wr = gauss_legendre(nq)
    xs, ws, es = [], [], []
    uniq = np.unique(t)
    for e in range(len(uniq) - 1):
        a, b = uniq[e], uniq[e + 1]
        xs.append(a + (b - a) * xr)
        ws.append((b - a) * wr)
        es.append(np.full(nq, e))
    return np.concatenate(xs), np.concatenate(ws), np.concatenate(es)


def mass_stiffness_1d(t: np.ndarray, p: int):
    """Univariate M_ij = int_0^1 B_i B_j and K_ij = int_0^1 B_i' B_j' (exact: p+1 Gauss
    points per interval integrate degree 2p+1)."""
    x, w, _ = quadrature_points(t, p)
    B = basis(t, p, x)
    dB = basis(t, p, x, 1)
    return B.T @ (w[:, None] * B), dB.T @ (w[:, None] * dB)


def insert_knot_matrix(t: np.ndarray, p: int, xbar: float):
    """Boehm's algorithm: coefficients c (n) of a spline on knots t map to c' (n+1) on
    t + {xbar} by c'_i = a_i c_i + (1 - a_i) c_{i-1}, a_i = (xbar - t_i)/(t_{i+p} - t_i)
    for mu-p+1 <= i <= mu (t_mu <= xbar < t_{mu+1}), c'_i = c_i below and c_{i-1} above.
    Returns (T, t') with c' = T c."""
    n = len(t) - p - 1
    mu = int(np.searchsorted(t, xbar, side="right") - 1)
    T = np.zeros((n + 1, n))
    for i in range(n + 1):
        if i <= mu - p:
            T[i, i] = 1.0
        elif i >= mu + 1:
            T[i, i - 1] = 1.0
        else:
            a = (xbar - t[i]) / (t[i + p] - t[i])
            T[i, i] = a
            T[i, i - 1] = 1.0 - a
    return T, np.sort(np.concatenate([t, [xbar]]))


def prolongation_1d(m_coarse: int, p: int) -> np.ndarray:
    """Matrix of the canonical embedding S_{p,1/m} -> S_{p,1/(2m)} (Sec. 3): insert every
    midpoint (2i+1)/(2m) once by Boehm's algorithm and multiply the single-knot steps."""
    t = uniform_knots(m_coarse, p)
    P = np.eye(m_coarse + p)
    for i in range(m_coarse):
        T, t = insert_knot_matrix(t, p, (2 * i + 1) / (2 * m_coarse))
        P = T @ P
    return P
