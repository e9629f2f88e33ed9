"""Grid hierarchy, the multigrid cycle of Algorithm 1 and PCG (Sec. 3, Sec. 4), on
globally assembled CSR matrices as in the paper's serial code.

Multigrid(l, u, f) (Algorithm 1, single address space so Sigma and chi are identities):
    nu times:  u <- u + tau L_l^{-1} (f - A_l u)                  (pre-smoothing, Eq. sm)
    r <- P_l^T (f - A_l u)
    l == 1:    p <- A_0^{-1} r                                     (exact coarse solve)
    else:      p <- 0; mu times p <- Multigrid(l-1, p, r)
    u <- u + P_l p           (undamped, as in Algorithm 1; Sec. 3 prints a tau here too)
    nu times:  u <- u + tau L_l^{-1} (f - A_l u)                  (post-smoothing)
With L = 0 (a single level) the preconditioner is A_0^{-1}.

PCG (Sec. 4, Sec. 5): standard preconditioned CG, one cycle from a zero initial guess per
iteration, stopped when ||b - A x_k||_2 <= tol ||b - A x_0||_2 (checked after every update).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import multipatch, smoother


@dataclass
class Level:
    space: multipatch.Space
    A: sp.csr_matrix
    P: Optional[sp.csr_matrix]          # V_{l-1} -> V_l (None on level 0)
    smooth: Optional[list]              # local smoothers (None on level 0)


@dataclass
class Hierarchy:
    levels: List[Level]
    coarse_chol: tuple
    tau: float = 0.25
    nu: int = 1
    mu: int = 1


def build_hierarchy(problem, tau=0.25, nu=1, mu=1) -> Hierarchy:
    levels = []
    prev = None
    for l in range(problem.num_levels):
        sp_l = multipatch.build_space(problem, l)
        A = multipatch.stiffness(problem, sp_l)
        P = multipatch.prolongation(prev, sp_l) if prev is not None else None
        sm = smoother.build_smoother(sp_l, l) if l > 0 else None
        levels.append(Level(sp_l, A, P, sm))
        prev = sp_l
    A0 = levels[0].A.toarray()
    return Hierarchy(levels, sla.cho_factor(A0, lower=True), tau, nu, mu)


def multigrid(H: Hierarchy, l: int, u: np.ndarray, f: np.ndarray) -> np.ndarray:
    if l == 0:
        return sla.cho_solve(H.coarse_chol, f)
    lv = H.levels[l]
    for _ in range(H.nu):
        u = u + H.tau * smoother.apply_smoother(lv.smooth, f - lv.A @ u)
    r = lv.P.T @ (f - lv.A @ u)
    if l == 1:
        p = sla.cho_solve(H.coarse_chol, r)
    else:
        p = np.zeros(len(r))
        for _ in range(H.mu):
            p = multigrid(H, l - 1, p, r)
    u = u + lv.P @ p
    for _ in range(H.nu):
        u = u + H.tau * smoother.apply_smoother(lv.smooth, f - lv.A @ u)
    return u


def precondition(H: Hierarchy, r: np.ndarray) -> np.ndarray:
    L = len(H.levels) - 1
    return multigrid(H, L, np.zeros_like(r), r)


@dataclass
class PCGResult:
    x: np.ndarray
    iters: int
    relres: float
    history: list


def pcg(H: Hierarchy, b: np.ndarray, x0=None, tol=1e-8, max_iter=500, fixed_iters=None):
    """Preconditioned CG; `fixed_iters` runs exactly that many iterations."""
    A = H.levels[-1].A
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A @ x
    r0 = np.linalg.norm(r)
    hist = [1.0]
    if r0 == 0.0:
        return PCGResult(x, 0, 0.0, hist)
    z = precondition(H, r)
    p = z.copy()
    rz = r @ z
    it = 0
    while True:
        if fixed_iters is None and hist[-1] <= tol:
            break
        if fixed_iters is not None and it >= fixed_iters:
            break
        if it >= max_iter:
            break
        w = A @ p
        alpha = rz / (p @ w)
        x = x + alpha * p
        r = r - alpha * w
        it += 1
        hist.append(np.linalg.norm(r) / r0)
        if fixed_iters is None and hist[-1] <= tol:
            break
        z = precondition(H, r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return PCGResult(x, it, hist[-1], hist)


def direct_solve(A: sp.spmatrix, b: np.ndarray) -> np.ndarray:
    """u* = A^{-1} b by dense Cholesky (the plain definition of the discrete solution)."""
    return sla.cho_solve(sla.cho_factor(A.toarray(), lower=True), b)
