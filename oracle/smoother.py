"""Local smoothers of the additive Schwarz smoother L_l^{-1} = sum_T P_T L_T^{-1} P_T^T
(Sec. 3, Eq. additive).

Patch interiors -- subspace-corrected mass smoother.  The paper takes it from a cited work
that is not part of its text; the reading used here (stated once, used by both the
oracle and the CUDA library) is:

  per direction j of the interior index set I_j (ends dropped at interface/Dirichlet
  sides), split span{B_i : i in I_j} = S~ (+) S^G, where S~ holds the splines with
      D^r u(end) = 0 for odd r < p at every kept (Neumann) end and
      D^r u(end) = 0 for even r, 2 <= r < p, at every dropped end,
  and S^G is its M-orthogonal complement.  With an M-orthonormal basis U~ of S~ and
  the M-orthonormal generalized eigenvectors U^G of (K, M) on S^G (eigenvalues lam),
  Ubar = [U~, U^G] and mu = [sigma, ..., sigma, lam + sigma].  Then
      L_T^{-1} = (Ubar_0 x ... x Ubar_{d-1}) diag(1 / sum_j mu_j) (Ubar_0 x ...)^T
  with sigma = 5 h^{-2} (Sec. 5: sigma = h^{-2}/0.2), h = 1/m_l on the parameter domain.

Edges (2D, Sec. 3 list):  L_T = (h/p)^{d-1} K + (h/p)^{d-3} M on the edge's interior
indices (both ends dropped), so (h/p) K + (p/h) M in 2D and (h/p)^2 K + M in 3D.
Vertices:  L_T = (h/p)^{d-2}.
Faces (3D):  L*_T = (h/p)(K x M + M x K + (p/h)^2 M x M), applied as the subspace-corrected
mass smoother with the diagonal sum_j mu_j replaced by (h/p)(mu_0 + mu_1 + p^2/h^2).

K and M are the univariate matrices of Sec. 3 on the patch's knot vector; the constants
"spectrally equivalent" / "in the order of" are taken as 1.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Tuple

import numpy as np
import scipy.linalg as sla

from . import bspline
from .multipatch import Piece, Space

SIGMA_SCALE = 5.0


def end_derivatives(t: np.ndarray, p: int, r: int):
    """Row vectors D^r B_i(0) and D^r B_i(1) (one-sided) for all i."""
    return bspline.basis(t, p, [0.0], r)[0], bspline.basis(t, p, [1.0], r)[0]


def scms_1d(t: np.ndarray, p: int, drop_lo: bool, drop_hi: bool, sigma: float):
    key = (tuple(np.asarray(t).tolist()), int(p), bool(drop_lo), bool(drop_hi), float(sigma))
    if key not in _SCMS_CACHE:
        _SCMS_CACHE[key] = _scms_1d(t, p, drop_lo, drop_hi, sigma)
    return _SCMS_CACHE[key]


_SCMS_CACHE: dict = {}


def _scms_1d(t: np.ndarray, p: int, drop_lo: bool, drop_hi: bool, sigma: float):
    """(Ubar, mu) of the subspace-corrected mass smoother on one direction (reading in the
    module docstring).  Ubar is |I| x |I| with Ubar^T M_I Ubar = I."""
    M, K = bspline.mass_stiffness_1d(t, p)
    n = M.shape[0]
    I = np.arange(1 if drop_lo else 0, n - 1 if drop_hi else n)
    MI, KI = M[np.ix_(I, I)], K[np.ix_(I, I)]
    rows = []
    for end, dropped in ((0, drop_lo), (1, drop_hi)):
        orders = range(2, p, 2) if dropped else range(1, p, 2)
        for r in orders:
            lo, hi = end_derivatives(t, p, r)
            v = (lo if end == 0 else hi)[I]
            rows.append(v / np.max(np.abs(v)))
    C = np.array(rows).reshape(len(rows), len(I))
    Z = sla.null_space(C) if len(rows) else np.eye(len(I))
    Q = sla.orth(C.T) if len(rows) else np.zeros((len(I), 0))
    blocks, mus = [], []
    if Z.shape[1]:
        lam, Y = sla.eigh(Z.T @ KI @ Z, Z.T @ MI @ Z)
        blocks.append(Z @ Y)
        mus.append(np.full(Z.shape[1], sigma))
    if Q.shape[1]:
        W = np.linalg.solve(MI, Q)
        lam, Y = sla.eigh(W.T @ KI @ W, W.T @ MI @ W)
        blocks.append(W @ Y)
        mus.append(lam + sigma)
    return np.hstack(blocks), np.concatenate(mus), I


def fd_apply(Us: List[np.ndarray], Dinv: np.ndarray, R: np.ndarray) -> np.ndarray:
    """(U_0 x ... x U_{d-1}) diag(Dinv) (U_0 x ...)^T applied to the tensor R, via the
    Kronecker identity (U_0 x U_1) vec(R) = vec(U_0 R U_1^T), one mode at a time."""
    Y = R
    for j, U in enumerate(Us):
        Y = np.moveaxis(np.tensordot(U.T, Y, axes=([1], [j])), 0, j)
    Y = Y * Dinv
    for j, U in enumerate(Us):
        Y = np.moveaxis(np.tensordot(U, Y, axes=([1], [j])), 0, j)
    return Y


@dataclass
class LocalSmoother:
    piece: Piece
    Us: List[np.ndarray]       # FD bases per piece axis (empty for vertices)
    Dinv: np.ndarray           # tensor of 1/diagonal (scalar for vertices)
    dense_L: np.ndarray | None = None  # explicit L_T for small pieces (tests)


def build_smoother(space: Space, level: int, explicit: bool = False) -> List[LocalSmoother]:
    d = space.dim
    out = []
    for pc in space.pieces:
        k = pc.patch
        h = 1.0 / space.m[k, 0]
        p = int(space.p[k, 0])
        sigma = SIGMA_SCALE / h ** 2
        if pc.kind == "interior":
            Us, mus = [], []
            for j in range(d):
                U, mu, _ = scms_1d(space.knots[k][j], int(space.p[k, j]), *pc.drop[j],
                                   SIGMA_SCALE * space.m[k, j] ** 2)
                Us.append(U); mus.append(mu)
            D = sum(np.meshgrid(*mus, indexing="ij"))
            out.append(LocalSmoother(pc, Us, 1.0 / D))
        elif pc.kind == "vertex":
            out.append(LocalSmoother(pc, [], np.array(1.0 / (h / p) ** (d - 2))))
        elif pc.kind == "edge":
            j = pc.dirs[0]
            h, p = 1.0 / space.m[k, j], int(space.p[k, j])
            t = space.knots[k][j]
            M, K = bspline.mass_stiffness_1d(t, p)
            MI, KI = M[1:-1, 1:-1], K[1:-1, 1:-1]
            a, b = (h / p) ** (d - 1), (h / p) ** (d - 3)
            lam, U = sla.eigh(KI, MI)
            out.append(LocalSmoother(pc, [U], 1.0 / (a * lam + b),
                                     a * KI + b * MI if explicit else None))
        elif pc.kind == "face":
            Us, mus = [], []
            for j in pc.dirs:
                U, mu, _ = scms_1d(space.knots[k][j], p, True, True, sigma)
                Us.append(U); mus.append(mu)
            D = (h / p) * (sum(np.meshgrid(*mus, indexing="ij")) + p ** 2 / h ** 2)
            out.append(LocalSmoother(pc, Us, 1.0 / D))
    return out


def apply_smoother(smoothers: List[LocalSmoother], r: np.ndarray) -> np.ndarray:
    """z = L_l^{-1} r = sum_T P_T L_T^{-1} P_T^T r (block diagonal over pieces)."""
    z = np.zeros_like(r)
    for s in smoothers:
        ids = s.piece.ids
        if s.piece.kind == "vertex":
            z[ids] = s.Dinv * r[ids]
        else:
            z[ids] = fd_apply(s.Us, s.Dinv, r[ids])
    return z


def dense_local_operator(s: LocalSmoother) -> np.ndarray:
    """Explicit L_T = (Ubar^{-T} x ...) diag(D) (Ubar^{-1} x ...) of an FD-form smoother,
    for tests on tiny pieces."""
    Uk = np.ones((1, 1))
    for U in s.Us:
        Uk = np.kron(Uk, U)
    Uinv = np.linalg.inv(Uk)
    return Uinv.T @ np.diag(1.0 / np.ravel(s.Dinv)) @ Uinv
