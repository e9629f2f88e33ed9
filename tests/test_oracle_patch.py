"""Pins of the oracle's patch forms a_k (Eq. model:bil) against closed forms: the
parameter-domain Kronecker sum for axis-aligned affine patches, exact energies of linear
functions, the area of a bilinear quadrilateral, rigid-motion invariance."""
import numpy as np
import pytest

from oracle import bspline, patch


def quad_corners(pts):
    """Corners in the input order c = c_0 + 2 c_1 from a counter-clockwise list."""
    a, b, c, d = pts  # (0,0) (1,0) (1,1) (0,1) in parameter space
    return np.array([a, b, d, c], dtype=float)


def shoelace(pts):
    x, y = np.array(pts).T
    return 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))


def spline_fit(knots, p, fun_of_xi, dim):
    """Exact coefficients of a function that lies in the tensor spline space (least squares
    over the tensor Gauss points)."""
    xs = [bspline.quadrature_points(t, p)[0] for t in knots]
    Bs = [bspline.basis(t, p, x) for t, x in zip(knots, xs)]
    G = Bs[0]
    for B in Bs[1:]:
        G = np.kron(G, B)
    grid = np.stack([g.ravel() for g in np.meshgrid(*xs, indexing="ij")], axis=1)
    return np.linalg.lstsq(G, fun_of_xi(grid), rcond=None)[0]


@pytest.mark.parametrize("p,m", [(2, 3), (3, 4), (4, 2)])
def test_affine_square_is_kronecker_sum(p, m):
    t = bspline.uniform_knots(m, p)
    M, K = bspline.mass_stiffness_1d(t, p)
    for s, off in ((1.0, (0, 0)), (0.25, (3.0, -1.0))):
        pts = [(0, 0), (s, 0), (s, s), (0, s)]
        C = quad_corners(np.array(pts) + off)
        A = patch.patch_matrices(C, [t, t], [p, p]).toarray()
        np.testing.assert_allclose(A, np.kron(K, M) + np.kron(M, K), atol=1e-12)


def test_affine_cube_3d_scaling():
    p, m, s = 2, 2, 0.5
    t = bspline.uniform_knots(m, p)
    M, K = bspline.mass_stiffness_1d(t, p)
    bits = patch.corner_bits(3)
    C = bits * s
    A = patch.patch_matrices(C, [t, t, t], [p, p, p]).toarray()
    expect = s * (np.kron(np.kron(K, M), M) + np.kron(np.kron(M, K), M) + np.kron(np.kron(M, M), K))
    np.testing.assert_allclose(A, expect, atol=1e-12)


QUADS = [
    [(0, 0), (1, 0), (1, 1), (0, 1)],
    [(0.1, -0.05), (1.08, 0.02), (0.93, 1.1), (-0.04, 0.97)],
    [(0, 0), (2, 0.3), (1.6, 1.4), (0.2, 0.9)],
]


@pytest.mark.parametrize("pts", QUADS)
@pytest.mark.parametrize("p,m", [(2, 3), (4, 2)])
def test_linear_function_energy_and_area(pts, p, m):
    """u(x,y) = a.x + b lies in the space (u o G is bilinear), so c^T A c = |a|^2 area and
    A c_const = 0; 1^T M_geo 1 = area (shoelace)."""
    C = quad_corners(pts)
    t = bspline.uniform_knots(m, p)
    A, Mg = patch.patch_matrices(C, [t, t], [p, p], want_mass=True)
    area = shoelace(pts)
    one = np.ones(A.shape[0])
    np.testing.assert_allclose(one @ (Mg @ one), area, rtol=1e-13)
    np.testing.assert_allclose(A @ one, 0.0, atol=1e-12)
    a = np.array([0.7, -1.3])
    c = spline_fit([t, t], p, lambda xi: patch.geometry(C, xi)[0] @ a + 0.4, 2)
    np.testing.assert_allclose(c @ (A @ c), a @ a * area, rtol=1e-11)
    assert np.all(np.linalg.eigvalsh(A.toarray()) > -1e-10)
    np.testing.assert_allclose(A.toarray(), A.toarray().T, atol=1e-14)


def test_rigid_motion_invariance():
    p, m = 3, 3
    t = bspline.uniform_knots(m, p)
    C = quad_corners(QUADS[2])
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    A1 = patch.patch_matrices(C, [t, t], [p, p]).toarray()
    A2 = patch.patch_matrices(C @ R.T + np.array([5.0, -2.0]), [t, t], [p, p]).toarray()
    np.testing.assert_allclose(A1, A2, atol=1e-12)


def test_trilinear_linear_energy():
    p, m = 2, 2
    t = bspline.uniform_knots(m, p)
    rng = np.random.default_rng(5)
    C = patch.corner_bits(3).astype(float) + rng.uniform(-0.08, 0.08, (8, 3))
    A, Mg = patch.patch_matrices(C, [t, t, t], [p, p, p], want_mass=True)
    a = np.array([0.3, -0.8, 1.1])
    c = spline_fit([t, t, t], p, lambda xi: patch.geometry(C, xi)[0] @ a, 3)
    vol = np.ones(A.shape[0]) @ (Mg @ np.ones(A.shape[0]))
    np.testing.assert_allclose(c @ (A @ c), a @ a * vol, rtol=1e-11)


@pytest.mark.parametrize("dim,p,m", [(2, 3, 5), (3, 2, 3)])
def test_elementwise_bands_equal_kronecker_form(dim, p, m):
    t = bspline.uniform_knots(m, p)
    rng = np.random.default_rng(dim)
    C = patch.corner_bits(dim).astype(float) * 1.5 + rng.uniform(-0.1, 0.1, (2 ** dim, dim))
    A1, M1 = patch.patch_matrices(C, [t] * dim, [p] * dim, want_mass=True)
    A2 = patch.bands_to_csr(patch.patch_bands(C, [t] * dim, [p] * dim, chunk=7), [p] * dim)
    M2 = patch.bands_to_csr(patch.patch_bands(C, [t] * dim, [p] * dim, mass=True), [p] * dim)
    assert abs(A1 - A2).max() < 1e-14 * abs(A1).max() * 10
    assert abs(M1 - M2).max() < 1e-14 * abs(M1).max() * 10


@pytest.mark.parametrize("dim,p,m", [(2, 2, 3), (2, 4, 2), (3, 2, 2)])
def test_affine_mass_is_scaled_kronecker_product(dim, p, m):
    """An affine map G(xi) = x0 + J xi (sheared, not axis-aligned) has constant |det J|, so
    the geometry mass matrix is |det J| (M x ... x M) with the univariate mass matrix M of
    the knot vector (whose rows are pinned separately); both the Kronecker-form and the
    element-by-element (band) assembly must give it."""
    t = bspline.uniform_knots(m, p)
    M, _ = bspline.mass_stiffness_1d(t, p)
    rng = np.random.default_rng(11 + dim)
    J = np.eye(dim) * 1.3 + rng.uniform(-0.3, 0.3, (dim, dim))
    x0 = rng.uniform(-2, 2, dim)
    C = x0 + patch.corner_bits(dim).astype(float) @ J.T
    expect = abs(np.linalg.det(J)) * M
    for _ in range(dim - 1):
        expect = np.kron(expect, M)
    _, Mg = patch.patch_matrices(C, [t] * dim, [p] * dim, want_mass=True)
    Mb = patch.bands_to_csr(patch.patch_bands(C, [t] * dim, [p] * dim, mass=True), [p] * dim)
    np.testing.assert_allclose(Mg.toarray(), expect, atol=1e-14 * abs(expect).max() * 10)
    np.testing.assert_allclose(Mb.toarray(), expect, atol=1e-14 * abs(expect).max() * 10)


@pytest.mark.parametrize("p,m", [(2, 3), (3, 2)])
def test_bilinear_mass_entries_against_independent_quadrature(p, m):
    """Non-affine bilinear patch: every entry M_geo[(a,b),(c,d)] = int B_a B_c (xi0)
    B_b B_d (xi1) |det J(xi)| dxi, evaluated with SciPy's B-splines and a Gauss rule of its
    own on each element (|det J| is affine for a bilinear map, so the rule is exact) — a
    mix-up of basis indices in the oracle's element scatter would fail here."""
    from scipy.interpolate import BSpline
    t = bspline.uniform_knots(m, p)
    n = m + p
    C = quad_corners(QUADS[2])
    xg, wg = np.polynomial.legendre.leggauss(p + 2)
    xs, ws = [], []
    for e in range(m):
        a, b = e / m, (e + 1) / m
        xs.append(a + (b - a) * (xg + 1) / 2)
        ws.append((b - a) / 2 * wg)
    x1, w1 = np.concatenate(xs), np.concatenate(ws)
    B = np.stack([BSpline(t, np.eye(n)[i], p, extrapolate=False)(x1) for i in range(n)], axis=1)
    B = np.nan_to_num(B)
    X0, X1 = np.meshgrid(x1, x1, indexing="ij")
    W = np.outer(w1, w1)
    # Jacobian of the bilinear map written out (corner c = c0 + 2 c1 at xi = (c0, c1))
    d0 = (1 - X1)[..., None] * (C[1] - C[0]) + X1[..., None] * (C[3] - C[2])
    d1 = (1 - X0)[..., None] * (C[2] - C[0]) + X0[..., None] * (C[3] - C[1])
    dj = np.abs(d0[..., 0] * d1[..., 1] - d0[..., 1] * d1[..., 0]) * W
    expect = np.einsum("qa,qc,rb,rd,qr->abcd", B, B, B, B, dj).reshape(n * n, n * n)
    Mb = patch.bands_to_csr(patch.patch_bands(C, [t, t], [p, p], mass=True), [p, p]).toarray()
    _, Mg = patch.patch_matrices(C, [t, t], [p, p], want_mass=True)
    np.testing.assert_allclose(Mb, expect, atol=1e-13 * abs(expect).max())
    np.testing.assert_allclose(Mg.toarray(), expect, atol=1e-13 * abs(expect).max())
