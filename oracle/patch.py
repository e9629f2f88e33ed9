"""Multilinear geometry maps G_k: (0,1)^d -> Omega_k (Sec. 2) and the patch-local
Galerkin matrices of the forms a_k (Eq. model:bil):

    A_k[i, j] = sum over elements, sum over Gauss points of
                w |det J| (J^{-T} grad phi_i) . (J^{-T} grad phi_j),

written as A_k = sum_{a,b} G_a^T diag(w C_ab) G_b with C = |det J| J^{-1} J^{-T}, where
G_a is the (points x dofs) matrix of d/dxi_a of the tensor-product basis.  The mass
matrix with geometry (used for the load vector) is G^T diag(w |det J|) G.

Tile order: local dofs of a patch are numbered in C order over (i_0, ..., i_{d-1}),
direction d-1 fastest; Gauss points likewise.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import bspline


def corner_bits(dim: int):
    return np.array([[(c >> j) & 1 for j in range(dim)] for c in range(2 ** dim)])


def geometry(corners: np.ndarray, xi: np.ndarray):
    """Points G(xi) (Q,d) and Jacobians J[q,a,j] = dG_a/dxi_j (Q,d,d) of the multilinear
    map G(xi) = sum_c v_c prod_j phi_{c_j}(xi_j), phi_0 = 1-s, phi_1 = s."""
    dim = corners.shape[1]
    bits = corner_bits(dim)
    Q = xi.shape[0]
    X = np.zeros((Q, dim))
    J = np.zeros((Q, dim, dim))
    for c in range(2 ** dim):
        phi = np.where(bits[c][None, :] == 1, xi, 1.0 - xi)          # (Q,d)
        dphi = np.where(bits[c] == 1, 1.0, -1.0)                      # (d,)
        X += np.prod(phi, axis=1)[:, None] * corners[c][None, :]
        for j in range(dim):
            others = np.prod(np.delete(phi, j, axis=1), axis=1)
            J[:, :, j] += (dphi[j] * others)[:, None] * corners[c][None, :]
    return X, J


def _tensor_points(knots, p):
    """Per direction: Gauss points/weights of all elements."""
    return [bspline.quadrature_points(t, p) for t in knots]


def _kron_all(mats):
    out = sp.csr_matrix(mats[0])
    for M in mats[1:]:
        out = sp.kron(out, sp.csr_matrix(M), format="csr")
    return out


def patch_matrices(corners, knots, degrees, elem_window=None, want_mass=False):
    """Stiffness A_k (and optionally the geometry mass matrix) of one patch, as sparse
    (n x n) matrices with n = prod_j n_j, by Gauss quadrature with p+1 points per
    element and direction.  `elem_window` = list of (lo, hi) element ranges per direction
    restricts the quadrature to those elements (rows of dofs whose support lies inside the
    window are then exact)."""
    dim = len(knots)
    Bs, dBs, ws, xs = [], [], [], []
    for j in range(dim):
        x, w, e = bspline.quadrature_points(knots[j], int(degrees[j]))
        if elem_window is not None:
            lo, hi = elem_window[j]
            sel = (e >= lo) & (e < hi)
            x, w = x[sel], w[sel]
        Bs.append(bspline.basis(knots[j], int(degrees[j]), x))
        dBs.append(bspline.basis(knots[j], int(degrees[j]), x, 1))
        ws.append(w)
        xs.append(x)
    grids = np.meshgrid(*xs, indexing="ij")
    xi = np.stack([g.ravel() for g in grids], axis=1)
    wgrid = np.meshgrid(*ws, indexing="ij")
    W = np.prod(np.stack([g.ravel() for g in wgrid], axis=1), axis=1)
    _, J = geometry(corners, xi)
    detJ = np.linalg.det(J)
    Jinv = np.linalg.inv(J)
    C = np.abs(detJ)[:, None, None] * np.einsum("qai,qbi->qab", Jinv, Jinv)
    G = [_kron_all([dBs[j] if j == a else Bs[j] for j in range(dim)]) for a in range(dim)]
    A = None
    for a in range(dim):
        for b in range(dim):
            term = G[a].T @ sp.diags(W * C[:, a, b]) @ G[b]
            A = term if A is None else A + term
    A = A.tocsr()
    if not want_mass:
        return A
    G0 = _kron_all(Bs)
    Mg = (G0.T @ sp.diags(W * np.abs(detJ)) @ G0).tocsr()
    return A, Mg


def load_vector_analytic(corners, knots, degrees, f):
    """(f, phi_i)_{L2(Omega_k)} for an analytic source f(x) evaluated at the mapped Gauss
    points, same quadrature rule as the matrices."""
    dim = len(knots)
    Bs, ws, xs = [], [], []
    for j in range(dim):
        x, w, _ = bspline.quadrature_points(knots[j], int(degrees[j]))
        Bs.append(bspline.basis(knots[j], int(degrees[j]), x))
        ws.append(w)
        xs.append(x)
    grids = np.meshgrid(*xs, indexing="ij")
    xi = np.stack([g.ravel() for g in grids], axis=1)
    wgrid = np.meshgrid(*ws, indexing="ij")
    W = np.prod(np.stack([g.ravel() for g in wgrid], axis=1), axis=1)
    X, J = geometry(corners, xi)
    G0 = _kron_all(Bs)
    return G0.T @ (W * np.abs(np.linalg.det(J)) * f(X))


def _element_tables(t, p):
    """Per element e: Gauss points/weights and the values/derivatives of its p+1 non-zero
    B-splines B_e..B_{e+p} (open knot vector): shapes (m, p+1) and (m, p+1 q, p+1 a)."""
    x, w, e = bspline.quadrature_points(t, p)
    m = int(e.max()) + 1
    B = bspline.basis(t, p, x)
    dB = bspline.basis(t, p, x, 1)
    nq = p + 1
    T = np.zeros((m, nq, p + 1))
    dT = np.zeros((m, nq, p + 1))
    for el in range(m):
        rows = slice(el * nq, (el + 1) * nq)
        T[el] = B[rows, el:el + p + 1]
        dT[el] = dB[rows, el:el + p + 1]
    return x.reshape(m, nq), w.reshape(m, nq), T, dT


def patch_bands(corners, knots, degrees, chunk=4096, mass=False):
    """Element-by-element assembly of the same A_k (or of the geometry mass matrix): for
    each element the element matrix sum_{a,b} G_a^T diag(w C_ab) G_b over its Gauss points,
    scattered into the band storage band[i_0, ..., i_{d-1}, t] with t the flattened offset
    (j - i + p) in (2p+1)^d, i.e. A_k[i, j] = band[i, t(j - i)]."""
    dim = len(knots)
    ps = [int(q) for q in degrees]
    tabs = [_element_tables(knots[j], ps[j]) for j in range(dim)]
    ms = [tb[2].shape[0] for tb in tabs]
    ns = [ms[j] + ps[j] for j in range(dim)]
    width = [2 * q + 1 for q in ps]
    band = np.zeros(tuple(ns) + (int(np.prod(width)),))
    elems = np.array(list(np.ndindex(*ms)))
    nloc = [q + 1 for q in ps]
    loc = np.array(list(np.ndindex(*nloc)))          # local fn multi-indices (and qp ones)
    for s in range(0, len(elems), chunk):
        E = elems[s:s + chunk]
        nE = len(E)
        # qp coordinates, weights, and per-direction tables gathered per element
        xi = np.zeros((nE, len(loc), dim))
        W = np.ones((nE, len(loc)))
        Tv, Td = [], []
        for j in range(dim):
            xj, wj, T, dT = tabs[j]
            xi[:, :, j] = xj[E[:, j]][:, loc[:, j]]
            W *= wj[E[:, j]][:, loc[:, j]]
            Tv.append(T[E[:, j]]); Td.append(dT[E[:, j]])
        _, J = geometry(corners, xi.reshape(-1, dim))
        detJ = np.linalg.det(J)
        if mass:
            coef = (W.ravel() * np.abs(detJ)).reshape(nE, -1)
            G0 = np.ones((nE, len(loc), len(loc)))
            for j in range(dim):
                G0 *= Tv[j][:, loc[:, j]][:, :, loc[:, j]]
            Ae = np.matmul(G0.transpose(0, 2, 1), coef[:, :, None] * G0)
        else:
            Jinv = np.linalg.inv(J)
            C = (np.abs(detJ)[:, None, None] * np.einsum("qai,qbi->qab", Jinv, Jinv))
            C = C.reshape(nE, len(loc), dim, dim) * W[:, :, None, None]
            G = []
            for a in range(dim):
                Ga = np.ones((nE, len(loc), len(loc)))
                for j in range(dim):
                    tab = Td[j] if j == a else Tv[j]
                    Ga *= tab[:, loc[:, j]][:, :, loc[:, j]]
                G.append(Ga)
            Ae = np.zeros((nE, len(loc), len(loc)))
            for a in range(dim):
                for b in range(dim):
                    Ae += np.matmul(G[a].transpose(0, 2, 1), C[:, :, a, b, None] * G[b])
        for ia, la in enumerate(loc):
            rows = tuple(E[:, j] + la[j] for j in range(dim))
            for ib, lb in enumerate(loc):
                t = 0
                for j in range(dim):
                    t = t * width[j] + (lb[j] - la[j] + ps[j])
                band[rows + (np.full(nE, t),)] += Ae[:, ia, ib]   # rows distinct within a chunk
    return band


def bands_to_csr(band, degrees):
    """Sparse (n x n) matrix of a band array from `patch_bands` (tile C order)."""
    ns = band.shape[:-1]
    dim = len(ns)
    width = [2 * int(q) + 1 for q in degrees]
    idx = np.indices(ns).reshape(dim, -1)
    rows_all, cols_all, vals_all = [], [], []
    flat = band.reshape(-1, band.shape[-1])
    for t, off in enumerate(np.ndindex(*width)):
        tgt = idx + (np.array(off) - np.array([int(q) for q in degrees]))[:, None]
        ok = np.all((tgt >= 0) & (tgt < np.array(ns)[:, None]), axis=0)
        r = np.ravel_multi_index(idx[:, ok], ns)
        c = np.ravel_multi_index(tgt[:, ok], ns)
        rows_all.append(r); cols_all.append(c); vals_all.append(flat[r, t])
    n = int(np.prod(ns))
    return sp.csr_matrix((np.concatenate(vals_all),
                          (np.concatenate(rows_all), np.concatenate(cols_all))), shape=(n, n))
