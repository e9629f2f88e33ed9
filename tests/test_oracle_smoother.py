"""Pins of the oracle's local smoothers (Sec. 3) and of the transfer operators (Sec. 3,
Sec. 4).  The subspace-corrected mass smoother's fast-diagonalisation form is checked
against an eigenvector-free statement of the same operator (M-orthogonal projectors onto
S~ and S^G, per-subspace operators sigma M or K + sigma M); edge/face smoothers against
their explicitly assembled matrices."""
import itertools

import numpy as np
import pytest
import scipy.linalg as sla

import workloads
from oracle import bspline, multipatch, smoother, solver


def constraint_matrix(t, p, drop_lo, drop_hi):
    M, K = bspline.mass_stiffness_1d(t, p)
    n = M.shape[0]
    I = np.arange(1 if drop_lo else 0, n - 1 if drop_hi else n)
    rows = []
    for x, dropped in ((0.0, drop_lo), (1.0, drop_hi)):
        for r in (range(2, p, 2) if dropped else range(1, p, 2)):
            rows.append(bspline.basis(t, p, [x], r)[0][I])
    return np.array(rows).reshape(len(rows), len(I)), M[np.ix_(I, I)], K[np.ix_(I, I)]


CASES = [(p, m, lo, hi) for p in (2, 3, 4, 5) for m in (2, 5, 12)
         for lo, hi in itertools.product([False, True], repeat=2)]


@pytest.mark.parametrize("p,m,lo,hi", CASES)
def test_scms_basis_properties(p, m, lo, hi):
    t = bspline.uniform_knots(m, p)
    sigma = 5.0 * m * m
    U, mu, I = smoother.scms_1d(t, p, lo, hi, sigma)
    C, MI, KI = constraint_matrix(t, p, lo, hi)
    np.testing.assert_allclose(U.T @ MI @ U, np.eye(len(I)), atol=1e-9)
    assert np.all(mu >= sigma * (1 - 1e-12))
    ntilde = np.sum(np.isclose(mu, sigma, rtol=1e-12))
    if C.shape[0]:
        np.testing.assert_allclose(C @ U[:, :ntilde], 0.0, atol=1e-8 * np.abs(C).max())
    # the complement block is K-diagonal with eigenvalues mu - sigma
    UG = U[:, ntilde:]
    np.testing.assert_allclose(UG.T @ KI @ UG, np.diag(mu[ntilde:] - sigma),
                               atol=1e-8 * max(1.0, np.abs(KI).max()))


def projector_form(ts, ps, drops, sigma):
    """Eigenvector-free L: sum over alpha in {~,G}^d of Pi_alpha^T [sum_j M x..x X_j x..x M]
    Pi_alpha with X_j = sigma M_j on S~ and K_j + sigma M_j on S^G, Pi the M-orthogonal
    projectors (built from a null-space basis, no eigen decomposition)."""
    blocks = []
    for t, p, (lo, hi) in zip(ts, ps, drops):
        C, MI, KI = constraint_matrix(t, p, lo, hi)
        Z = sla.null_space(C) if C.shape[0] else np.eye(MI.shape[0])
        Pt = Z @ np.linalg.solve(Z.T @ MI @ Z, Z.T @ MI)       # onto S~ along S^G
        Pg = np.eye(MI.shape[0]) - Pt
        blocks.append((MI, KI, Pt, Pg))
    d = len(blocks)
    total = 0
    for alpha in itertools.product([0, 1], repeat=d):
        Pi = np.ones((1, 1))
        for j in range(d):
            Pi = np.kron(Pi, blocks[j][2] if alpha[j] == 0 else blocks[j][3])
        Lalpha = 0
        for j in range(d):
            term = np.ones((1, 1))
            for i in range(d):
                MI, KI = blocks[i][0], blocks[i][1]
                if i == j:
                    X = sigma * MI if alpha[i] == 0 else KI + sigma * MI
                else:
                    X = MI
                term = np.kron(term, X)
            Lalpha = Lalpha + term
        total = total + Pi.T @ Lalpha @ Pi
    return total


@pytest.mark.parametrize("p,m,drops", [
    (2, 4, [(True, True), (True, False)]),
    (3, 3, [(False, False), (True, True)]),
    (4, 2, [(True, False), (False, True)]),
    (4, 5, [(True, True), (True, True)]),
])
def test_fd_equals_projector_definition_2d(p, m, drops):
    t = bspline.uniform_knots(m, p)
    sigma = 5.0 * m * m
    Us, mus = [], []
    for lo, hi in drops:
        U, mu, _ = smoother.scms_1d(t, p, lo, hi, sigma)
        Us.append(U); mus.append(mu)
    D = sum(np.meshgrid(*mus, indexing="ij"))
    s = smoother.LocalSmoother(None, Us, 1.0 / D)
    L_fd = smoother.dense_local_operator(s)
    L_def = projector_form([t, t], [p, p], drops, sigma)
    np.testing.assert_allclose(L_fd, L_def, rtol=1e-9, atol=1e-9 * np.abs(L_def).max())
    x = np.random.default_rng(0).normal(size=D.shape)
    z = smoother.fd_apply(Us, 1.0 / D, x)
    np.testing.assert_allclose(L_def @ z.ravel(), x.ravel(), rtol=1e-9, atol=1e-9)


def test_fd_equals_projector_definition_3d():
    p, m = 2, 3
    t = bspline.uniform_knots(m, p)
    sigma = 5.0 * m * m
    drops = [(True, True), (False, True), (True, False)]
    Us, mus = [], []
    for lo, hi in drops:
        U, mu, _ = smoother.scms_1d(t, p, lo, hi, sigma)
        Us.append(U); mus.append(mu)
    D = sum(np.meshgrid(*mus, indexing="ij"))
    L_fd = smoother.dense_local_operator(smoother.LocalSmoother(None, Us, 1.0 / D))
    L_def = projector_form([t] * 3, [p] * 3, drops, sigma)
    np.testing.assert_allclose(L_fd, L_def, rtol=1e-9, atol=1e-9 * np.abs(L_def).max())


def test_edge_and_vertex_smoothers_2d():
    pr = workloads.perturbed_grid_2d(2, 3, 8, 4, 7)
    space = multipatch.build_space(pr, 3)
    sms = smoother.build_smoother(space, 3, explicit=True)
    h, p = 1.0 / 8, 3
    M, K = bspline.mass_stiffness_1d(bspline.uniform_knots(8, p), p)
    Le = (h / p) * K[1:-1, 1:-1] + (p / h) * M[1:-1, 1:-1]
    rng = np.random.default_rng(3)
    for s in sms:
        if s.piece.kind == "edge":
            np.testing.assert_allclose(s.dense_L, Le, rtol=1e-14)
            x = rng.normal(size=s.piece.ids.shape)
            z = smoother.fd_apply(s.Us, s.Dinv, x)
            np.testing.assert_allclose(Le @ z, x, rtol=1e-10, atol=1e-10)
        if s.piece.kind == "vertex":
            assert float(s.Dinv) == 1.0          # (h/p)^(d-2) = 1 in 2D


def test_face_smoother_3d():
    pr = workloads.perturbed_cube_3d(2, 2, 4, 3, 3)
    space = multipatch.build_space(pr, 2)
    sms = smoother.build_smoother(space, 2)
    h, p = 1.0 / 4, 2
    t = bspline.uniform_knots(4, p)
    faces = [s for s in sms if s.piece.kind == "face"]
    assert len(faces) == 12
    M, K = bspline.mass_stiffness_1d(t, p)
    MI = M[1:-1, 1:-1]
    L = (h / p) * (projector_form([t, t], [p, p], [(True, True)] * 2, 5.0 / h ** 2)
                   + (p / h) ** 2 * np.kron(MI, MI))
    Lfd = smoother.dense_local_operator(faces[0])
    np.testing.assert_allclose(Lfd, L, rtol=1e-9, atol=1e-9 * np.abs(L).max())
    edges = [s for s in sms if s.piece.kind == "edge"]
    assert len(edges) == 6
    x = np.random.default_rng(1).normal(size=edges[0].piece.ids.shape)
    Le = (h / p) ** 2 * K[1:-1, 1:-1] + MI
    np.testing.assert_allclose(Le @ smoother.fd_apply(edges[0].Us, edges[0].Dinv, x), x,
                               rtol=1e-10, atol=1e-10)
    verts = [s for s in sms if s.piece.kind == "vertex"]
    assert len(verts) == 1 and np.isclose(float(verts[0].Dinv), p / h)


def test_piece_partition_covers_all_dofs():
    pr = workloads.perturbed_cube_3d(2, 3, 4, 3, 3)
    space = multipatch.build_space(pr, 2)
    ids = np.concatenate([pc.ids.ravel() for pc in space.pieces])
    assert np.array_equal(np.sort(ids), np.arange(space.N))


# ---- transfers -------------------------------------------------------------------------

def test_prolongation_block_triangular_2d():
    """Sec. 4: a prolonged vertex value is the coarse vertex value; edge values depend on
    the edge and its vertices only; interiors on anything adjacent."""
    pr = workloads.perturbed_grid_2d(3, 3, 4, 3, 9)
    sc = multipatch.build_space(pr, 1)
    sf = multipatch.build_space(pr, 2)
    P = multipatch.prolongation(sc, sf).toarray()
    def piece_of(space):
        lab = {}
        for i, pc in enumerate(space.pieces):
            for g in pc.ids.ravel():
                lab[int(g)] = (pc.kind, i)
        return lab
    lf, lc = piece_of(sf), piece_of(sc)
    vert_c = {tuple(sorted(map(int, pc.ids.ravel()))) for pc in sc.pieces if pc.kind == "vertex"}
    for I in range(sf.N):
        kind, _ = lf[I]
        cols = np.nonzero(np.abs(P[I]) > 1e-15)[0]
        kinds = {lc[int(c)][0] for c in cols}
        if kind == "vertex":
            assert len(cols) == 1 and lc[int(cols[0])][0] == "vertex" and abs(P[I, cols[0]] - 1) < 1e-15
        if kind == "edge":
            assert kinds <= {"edge", "vertex"}
            assert len({lc[int(c)][1] for c in cols if lc[int(c)][0] == "edge"}) <= 1


def test_galerkin_identity_affine():
    pr = workloads.unit_square_quadrants(8, 3, 4)
    H = solver.build_hierarchy(pr)
    for l in range(1, 4):
        A_f, A_c, P = H.levels[l].A, H.levels[l - 1].A, H.levels[l].P
        G = (P.T @ A_f @ P).toarray()
        np.testing.assert_allclose(G, A_c.toarray(), atol=1e-12 * abs(A_c).max())


def test_prolongation_reproduces_multipatch_functions():
    pr = workloads.perturbed_cube_3d(2, 2, 4, 3, 3)
    sc = multipatch.build_space(pr, 1)
    sf = multipatch.build_space(pr, 2)
    P = multipatch.prolongation(sc, sf)
    uc = np.random.default_rng(0).normal(size=sc.N)
    uf = P @ uc
    x = np.random.default_rng(1).uniform(0, 1, (50, 3))
    for k in range(pr.num_patches):
        def eval_patch(space, u):
            cf = np.where(space.l2g[k] >= 0, u[np.maximum(space.l2g[k], 0)], 0.0)
            Bs = [bspline.basis(space.knots[k][j], 2, x[:, j]) for j in range(3)]
            return np.einsum("qa,qb,qc,abc->q", Bs[0], Bs[1], Bs[2], cf)
        np.testing.assert_allclose(eval_patch(sf, uf), eval_patch(sc, uc), atol=1e-13)
