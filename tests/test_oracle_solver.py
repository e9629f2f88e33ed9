"""Pins of the oracle's multigrid cycle (Algorithm 1) and PCG against what the mathematics
fixes: an exact coarse solve gives one-step convergence, tight PCG equals the dense
Cholesky solution, the V(1,1) preconditioner is symmetric positive definite, the
discretisation converges at order p+1 in L2 and p in H1 for a manufactured solution,
and the cycle's contraction stays bounded under refinement and degree elevation (the
robustness reported in Tables I and II)."""
import numpy as np
import pytest

import workloads
from oracle import bspline, multipatch, patch, solver


def sin_rhs(pr, space, scale=2 * np.pi ** 2):
    f = lambda X: scale * np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1])
    vecs = [patch.load_vector_analytic(np.asarray(pr.corners[k]), space.knots[k], space.p[k], f)
            for k in range(pr.num_patches)]
    return multipatch.global_vector(space, vecs)


def test_single_level_is_exact():
    pr = workloads.perturbed_grid_2d(2, 3, 1, 1, 4)
    H = solver.build_hierarchy(pr)
    b = np.random.default_rng(0).normal(size=H.levels[-1].space.N)
    res = solver.pcg(H, b, tol=1e-12)
    assert res.iters == 1 and res.relres < 1e-12


@pytest.mark.parametrize("maker", [
    lambda: workloads.unit_square_quadrants(8, 2, 4),
    lambda: workloads.perturbed_grid_2d(2, 4, 4, 3, 6),
    lambda: workloads.perturbed_cube_3d(2, 2, 4, 3, 3),
])
def test_tight_pcg_equals_direct_solve(maker):
    pr = maker()
    H = solver.build_hierarchy(pr)
    A = H.levels[-1].A
    b = np.random.default_rng(1).normal(size=A.shape[0])
    x = solver.pcg(H, b, tol=1e-13, max_iter=200).x
    xs = solver.direct_solve(A, b)
    assert np.linalg.norm(x - xs) <= 1e-10 * np.linalg.norm(xs)
    assert np.linalg.norm(b - A @ xs) <= 1e-13 * np.linalg.norm(b)


@pytest.mark.parametrize("maker", [
    lambda: workloads.perturbed_grid_2d(2, 3, 8, 4, 6),
    lambda: workloads.perturbed_cube_3d(2, 2, 4, 3, 3),
])
def test_preconditioner_symmetric_positive(maker):
    pr = maker()
    H = solver.build_hierarchy(pr)
    N = H.levels[-1].space.N
    rng = np.random.default_rng(2)
    X = rng.normal(size=(N, 3))
    BX = np.stack([solver.precondition(H, X[:, i]) for i in range(3)], axis=1)
    G = X.T @ BX
    np.testing.assert_allclose(G, G.T, rtol=1e-12, atol=1e-12 * np.abs(G).max())
    assert np.all(np.diag(G) > 0)


def l2_h1_errors(pr, space, u, exact, grad_exact):
    e2, g2 = 0.0, 0.0
    for k in range(pr.num_patches):
        kn, p = space.knots[k], int(space.p[k, 0])
        qs = [bspline.quadrature_points(t, p) for t in kn]
        B = [bspline.basis(t, p, q[0]) for t, q in zip(kn, qs)]
        dB = [bspline.basis(t, p, q[0], 1) for t, q in zip(kn, qs)]
        c = np.where(space.l2g[k] >= 0, u[np.maximum(space.l2g[k], 0)], 0.0)
        uh = B[0] @ c @ B[1].T
        d0 = dB[0] @ c @ B[1].T
        d1 = B[0] @ c @ dB[1].T
        xi = np.stack([g.ravel() for g in np.meshgrid(qs[0][0], qs[1][0], indexing="ij")], 1)
        W = np.outer(qs[0][1], qs[1][1]).ravel()
        X, J = patch.geometry(np.asarray(pr.corners[k]), xi)
        det = np.abs(np.linalg.det(J))
        grad_ref = np.stack([d0.ravel(), d1.ravel()], 1)
        grad = np.einsum("qji,qj->qi", np.linalg.inv(J), grad_ref)   # J^{-T} grad_ref
        e2 += np.sum(W * det * (uh.ravel() - exact(X)) ** 2)
        g2 += np.sum(W * det * np.sum((grad - grad_exact(X)) ** 2, axis=1))
    return np.sqrt(e2), np.sqrt(g2)


@pytest.mark.parametrize("p", [2, 3, 4])
def test_manufactured_solution_rates(p):
    """u = sin(pi x) sin(pi y) on the quadrant workload: L2 rate -> p+1, H1 rate -> p."""
    ex = lambda X: np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1])
    gex = lambda X: np.pi * np.stack([np.cos(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1]),
                                      np.sin(np.pi * X[:, 0]) * np.cos(np.pi * X[:, 1])], 1)
    errs = []
    for m in (2, 4, 8, 16):
        pr = workloads.unit_square_quadrants(m, p, int(np.log2(m)) + 1)
        H = solver.build_hierarchy(pr)
        sp_ = H.levels[-1].space
        res = solver.pcg(H, sin_rhs(pr, sp_), tol=1e-13, max_iter=300)
        errs.append(l2_h1_errors(pr, sp_, res.x, ex, gex))
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    assert rates[-1, 0] >= p + 1 - 0.2, rates
    assert rates[-1, 1] >= p - 0.2, rates


def contraction(H, iters=25, seed=0):
    """Spectral radius of the stationary iteration e <- (I - B A) e by power iteration."""
    A = H.levels[-1].A
    e = np.random.default_rng(seed).normal(size=A.shape[0])
    e /= np.linalg.norm(e)
    rho = 0.0
    for _ in range(iters):
        e_new = e - solver.precondition(H, A @ e)
        rho = np.linalg.norm(e_new)
        e = e_new / rho
    return rho


def test_contraction_bounded_in_h_and_p():
    """The V(1,1) contraction rises on the first levels, then saturates below 0.9 at the
    same value for every degree (robust in h and p)."""
    rhos = {}
    for p in (2, 4, 5):
        for lev in (5, 6, 7):
            pr = workloads.perturbed_grid_2d(2, p, 2 ** (lev - 1), lev, 8)
            rhos[(p, lev)] = contraction(solver.build_hierarchy(pr), iters=40)
    assert max(rhos.values()) < 0.9, rhos
    for p in (2, 4, 5):
        assert rhos[(p, 7)] - rhos[(p, 6)] < 0.01, rhos
    finest = [rhos[(p, 7)] for p in (2, 4, 5)]
    assert max(finest) - min(finest) < 0.02, rhos


def test_iteration_counts_band():
    its = []
    for p in (2, 4):
        for m, lev in ((8, 4), (32, 6)):
            pr = workloads.perturbed_grid_2d(4, p, m, lev, 2)
            H = solver.build_hierarchy(pr)
            b = workloads.rhs_coefficients(H.levels[-1].space.N, 2)
            its.append(solver.pcg(H, b, tol=1e-8).iters)
    assert all(10 <= i <= 60 for i in its), its
    assert max(its) - min(its) <= 10, its


@pytest.mark.parametrize("mu,nu", [(1, 1), (2, 1), (2, 2)])
def test_cycle_error_propagation_recursion(mu, nu):
    """Algorithm 1 as an iteration on A_l u = f has the error propagation
        E_l = S_l^nu (I - P_l (I - E_{l-1}^mu) A_{l-1}^{-1} P_l^T A_l) S_l^nu,  E_0 = 0,
    with S_l = I - tau B_l A_l (B_l the additive smoother): mu cycles from zero on the
    coarse residual equation leave (I - E^mu) A^{-1} r.  The oracle's cycle, applied to the
    unit vectors with f = 0, must give these dense matrices on every level (V- and W-cycle,
    one and two smoothing steps)."""
    from oracle import smoother as osm
    pr = workloads.perturbed_grid_2d(2, 2, 8, 4, 5)
    H = solver.build_hierarchy(pr, nu=nu, mu=mu)
    E_prev = None
    for l in range(1, len(H.levels)):
        lv = H.levels[l]
        A = lv.A.toarray()
        n = A.shape[0]
        I = np.eye(n)
        B = np.stack([osm.apply_smoother(lv.smooth, I[:, i]) for i in range(n)], axis=1)
        S = np.linalg.matrix_power(I - H.tau * B @ A, nu)
        Ac = H.levels[l - 1].A.toarray()
        P = lv.P.toarray()
        Q = np.eye(Ac.shape[0]) if l == 1 else np.eye(Ac.shape[0]) - np.linalg.matrix_power(E_prev, mu)
        E = S @ (I - P @ Q @ np.linalg.solve(Ac, P.T @ A)) @ S
        E_orc = np.stack([solver.multigrid(H, l, I[:, i], np.zeros(n)) for i in range(n)], axis=1)
        np.testing.assert_allclose(E_orc, E, rtol=0, atol=1e-11 * max(1.0, np.abs(E).max()), err_msg=f"level {l}")
        E_prev = E
    # a W-cycle contracts at least as well as a V-cycle here (spectral radius)
    if mu == 2 and nu == 1:
        HV = solver.build_hierarchy(pr, nu=1, mu=1)
        n = HV.levels[-1].A.shape[0]
        EV = np.stack([solver.multigrid(HV, len(HV.levels) - 1, np.eye(n)[:, i], np.zeros(n)) for i in range(n)],
                      axis=1)
        assert np.max(np.abs(np.linalg.eigvals(E_prev))) <= np.max(np.abs(np.linalg.eigvals(EV))) + 1e-12


@pytest.mark.parametrize("maker", [
    lambda: workloads.perturbed_grid_2d(2, 3, 8, 4, 6),
    lambda: workloads.perturbed_cube_3d(2, 2, 4, 3, 3),
])
def test_pcg_iterates_minimise_energy_error_over_krylov_space(maker):
    """With an SPD preconditioner B, the k-th PCG iterate from x_0 = 0 is the minimiser of
    ||x - A^{-1} b||_A over span{B b, (BA) B b, ..., (BA)^{k-1} B b}: the projected system
    V^T A V y = V^T b on an orthonormal basis V of that space gives it directly."""
    pr = maker()
    H = solver.build_hierarchy(pr)
    A = H.levels[-1].A
    N = A.shape[0]
    b = np.random.default_rng(8).uniform(-1, 1, N)
    K = [solver.precondition(H, b)]
    for k in range(1, 5):
        K.append(solver.precondition(H, A @ K[-1]))
    for k in range(1, 6):
        V, _ = np.linalg.qr(np.stack(K[:k], axis=1))
        y = np.linalg.solve(V.T @ (A @ V), V.T @ b)
        x_opt = V @ y
        x_k = solver.pcg(H, b, fixed_iters=k).x
        assert np.linalg.norm(x_k - x_opt) <= 1e-8 * np.linalg.norm(x_opt), k
