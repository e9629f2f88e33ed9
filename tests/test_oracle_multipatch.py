"""Pins of the oracle's multi-patch space (Eq. vh, Eq. matching, Eq. additive): the dof
counts printed in Table II for the Fichera corner, the sizes of the synthetic workloads,
constants/linear functions glued across interfaces (any gluing or orientation error breaks
them), invariance under re-parametrising a patch, and the piece partition."""
import os

import numpy as np
import pytest
import scipy.linalg as sla

import workloads
from oracle import multipatch, patch, bspline


def table2_rows():
    """Rows of tests/golden/fichera_table2.txt (values printed in Sec. 5.2, Table II)."""
    path = os.path.join(os.path.dirname(__file__), "golden", "fichera_table2.txt")
    rows = []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        split, p, m, levels, dofs, iters = line.split()
        rows.append((int(split), int(p), int(m), int(levels), None if dofs == "-" else int(dofs),
                     None if iters == "-" else int(iters)))
    return rows


@pytest.mark.parametrize("split,p,m,levels,expect", [r[:5] for r in table2_rows() if r[4] is not None])
def test_fichera_dof_counts_of_the_paper(split, p, m, levels, expect):
    pr = workloads.fichera_corner(split, p, m, levels)
    assert pr.num_patches == 7 * split ** 3
    assert multipatch.build_space(pr, levels - 1).N == expect


def test_workload_sizes():
    assert multipatch.build_space(workloads.unit_square_quadrants(), 3).N == 289
    s = multipatch.build_space(workloads.perturbed_grid_2d(4, 4, 256, 9, 2), 8)
    assert s.N == 1_073_296
    s0 = multipatch.build_space(workloads.perturbed_grid_2d(4, 4, 256, 9, 2), 0)
    assert s0.N == 256


def all_neumann(pr):
    pr.side_bc = np.where(pr.side_bc == 0, 0, 2)
    return pr


def fit_global(pr, space, fun):
    """Global coefficients of a physical function that lies in V (least squares per patch,
    then read through the dof map; the copies of a shared dof must agree)."""
    u = np.full(space.N, np.nan)
    for k in range(pr.num_patches):
        kn = space.knots[k]
        xs = [np.linspace(0, 1, 3 * (len(t))) for t in kn]
        Bs = [bspline.basis(t, int(space.p[k, j]), x) for j, (t, x) in enumerate(zip(kn, xs))]
        G = Bs[0]
        for B in Bs[1:]:
            G = np.kron(G, B)
        grid = np.stack([g.ravel() for g in np.meshgrid(*xs, indexing="ij")], axis=1)
        X, _ = patch.geometry(np.asarray(pr.corners[k]), grid)
        c = np.linalg.lstsq(G, fun(X), rcond=None)[0]
        g = space.l2g[k].ravel()
        prev = u[g]
        seen = ~np.isnan(prev)
        np.testing.assert_allclose(prev[seen], c[seen], atol=1e-10)
        u[g] = c
    return u


@pytest.mark.parametrize("maker", [
    lambda: all_neumann(workloads.perturbed_grid_2d(3, 2, 4, 2, 11)),
    lambda: all_neumann(workloads.perturbed_grid_2d(2, 3, 2, 2, 12)),
    lambda: all_neumann(workloads.perturbed_cube_3d(2, 2, 2, 2, 13)),
])
def test_glued_constants_and_linear_energy(maker):
    pr = maker()
    space = multipatch.build_space(pr, pr.num_levels - 1)
    A, Mg = multipatch.stiffness(pr, space, want_mass=True)
    one = np.ones(space.N)
    np.testing.assert_allclose(A @ one, 0.0, atol=1e-11)
    vol = one @ (Mg @ one)
    a = np.array([0.6, -1.1, 0.4][:pr.dim])
    u = fit_global(pr, space, lambda X: X @ a + 0.3)
    np.testing.assert_allclose(u @ (A @ u), (a @ a) * vol, rtol=1e-10)


def test_domain_volume_is_preserved():
    pr = all_neumann(workloads.perturbed_grid_2d(4, 2, 2, 2, 2))
    space = multipatch.build_space(pr, 1)
    _, Mg = multipatch.stiffness(pr, space, want_mass=True)
    one = np.ones(space.N)
    np.testing.assert_allclose(one @ (Mg @ one), 16.0, rtol=1e-13)   # [0,4]^2
    pr3 = all_neumann(workloads.perturbed_cube_3d(2, 2, 2, 2, 3))
    s3 = multipatch.build_space(pr3, 1)
    _, M3 = multipatch.stiffness(pr3, s3, want_mass=True)
    np.testing.assert_allclose(np.ones(s3.N) @ (M3 @ np.ones(s3.N)), 1.0, rtol=1e-13)


def reversed_patch(pr, k, direction):
    """Same geometry, patch k parametrised with direction `direction` reversed."""
    pr2 = workloads.Problem(pr.dim, pr.degree.copy(), pr.knots, pr.corners.copy(),
                            pr.side_bc.copy(), pr.num_levels)
    for c in range(2 ** pr.dim):
        pr2.corners[k, c] = pr.corners[k, c ^ (1 << direction)]
    s = 2 * direction
    pr2.side_bc[k, s], pr2.side_bc[k, s + 1] = pr.side_bc[k, s + 1], pr.side_bc[k, s]
    return pr2


@pytest.mark.parametrize("dim", [2, 3])
def test_orientation_invariance(dim):
    """Reversing a patch's parametrisation must give the same discrete problem up to a
    permutation: same N, same spectrum, and the same solution at the same dofs."""
    pr = (workloads.perturbed_grid_2d(2, 3, 2, 2, 21) if dim == 2
          else workloads.perturbed_cube_3d(2, 2, 2, 2, 22))
    pr2 = reversed_patch(pr, 1, 0)
    s1 = multipatch.build_space(pr, 1)
    s2 = multipatch.build_space(pr2, 1)
    assert s1.N == s2.N
    A1 = multipatch.stiffness(pr, s1).toarray()
    A2 = multipatch.stiffness(pr2, s2).toarray()
    np.testing.assert_allclose(np.linalg.eigvalsh(A1), np.linalg.eigvalsh(A2), rtol=1e-11, atol=1e-12)
    # map dofs: reversed local index of patch 1
    perm = np.full(s1.N, -1)
    for k in range(pr.num_patches):
        g1 = s1.l2g[k]
        g2 = s2.l2g[k] if k != 1 else np.flip(s2.l2g[k], axis=0)
        perm[g1[g1 >= 0]] = g2[g1 >= 0]
    assert np.all(np.sort(perm) == np.arange(s1.N))
    np.testing.assert_allclose(A2[np.ix_(perm, perm)], A1, atol=1e-12)


def test_pieces_and_dirichlet_cfg1():
    pr = workloads.unit_square_quadrants(8, 2, 4)
    s = multipatch.build_space(pr, 3)
    kinds = sorted(pc.kind for pc in s.pieces)
    assert kinds == ["edge"] * 4 + ["interior"] * 4 + ["vertex"]
    for pc in s.pieces:
        if pc.kind == "interior":
            assert pc.ids.shape == (8, 8)       # n = 10, both ends dropped
        if pc.kind == "edge":
            assert pc.ids.shape == (8,)
    A = multipatch.stiffness(pr, s)
    sla.cholesky(A.toarray())                   # SPD after Dirichlet elimination


def test_pieces_neumann_sides_stay_in_interior():
    pr = workloads.perturbed_grid_2d(2, 2, 4, 3, 5)   # D on x=0,y=0; N on x=4,y=4
    s = multipatch.build_space(pr, 2)
    sizes = {pc.patch: pc.ids.shape for pc in s.pieces if pc.kind == "interior"}
    n = 4 + 2
    assert sizes[0] == (n - 2, n - 2)
    assert sizes[3] == (n - 1, n - 1)             # Neumann ends kept
    assert sizes[1] == (n - 2, n - 1)
    nv = sum(pc.kind == "vertex" for pc in s.pieces)
    assert nv == 3                                # centre + two Neumann-boundary vertices
