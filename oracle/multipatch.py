"""Fully matching multi-patch space V_l (Eq. vh, Eq. matching) and its pieces.

Dofs.  Every patch k carries the full tensor basis of S_{p,h}; a basis function whose
node lies on a patch side, edge or vertex shared with other patches is glued with the
coinciding functions of those patches into one global C^0 dof (Sec. 2, Fig. 1: "a node
within one edge vanishes outside the union of that edge and the adjacent patches").
A node is identified across patches by the corner vertices of the smallest cube entity
(side / edge / vertex) containing it plus its index along that entity, measured from the
entity corner with the smallest global vertex id; the entity axes are ordered by the
vertex id of the neighbouring corner.  Dofs on the closure of a Dirichlet side of any
owner are eliminated (u = 0 on Gamma_D, Sec. 2).

Pieces (Eq. additive, Sec. 3, Fig. 2; reading: a node with a single owner belongs to
that patch's interior piece, Neumann-side nodes included; a node with several owners
belongs to the piece of the smallest shared entity: edge (2D) / face, edge (3D) /
vertex).  The patch-interior piece is the tensor set I_0 x ... x I_{d-1} where I_j drops
an end exactly when that side is an interface or Dirichlet.

Global numbering (oracle's own): scan patches in order, local nodes in tile (C) order;
a new id is given at the first occurrence of every non-Dirichlet node.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Tuple

import numpy as np
import scipy.sparse as sp

from . import bspline, patch

AUTO, DIRICHLET, NEUMANN, INTERFACE = 0, 1, 2, 3


@dataclass
class Piece:
    kind: str                 # "interior", "face", "edge", "vertex"
    ids: np.ndarray           # global dof ids, shaped as the piece's tensor (or 1 value)
    patch: int                # owner patch used for the 1D data
    dirs: Tuple[int, ...]     # patch-local directions of the piece axes (in id order)
    drop: Tuple[Tuple[bool, bool], ...] = ()  # for interiors: dropped (lo, hi) ends per dir


@dataclass
class Space:
    dim: int
    n: np.ndarray                    # (K, d) 1D basis sizes
    m: np.ndarray                    # (K, d) intervals
    p: np.ndarray                    # (K, d) degrees
    knots: List[List[np.ndarray]]
    l2g: List[np.ndarray]            # per patch: tile-shaped global ids, -1 = Dirichlet
    N: int
    side_type: np.ndarray            # (K, 2d) resolved: DIRICHLET/NEUMANN/INTERFACE
    pieces: List[Piece] = field(default_factory=list)


def vertex_ids(corners: np.ndarray, tol: float = 1e-9):
    """Global ids of patch corners: coordinates snapped to a grid of spacing tol * scale,
    then equal snapped coordinates are the same vertex (ids in order of first use)."""
    K, nc, d = corners.shape
    pts = corners.reshape(-1, d)
    scale = max(1.0, float(np.abs(pts).max()))
    snapped = np.round(pts / (tol * scale)).astype(np.int64)
    _, first, inv = np.unique(snapped, axis=0, return_index=True, return_inverse=True)
    order = np.argsort(np.argsort(first))          # renumber by first occurrence
    return order[inv.ravel()].reshape(K, nc)


def _entity_corners(dim, fixed):
    """Local corner indices of the cube entity with fixed {dir: end}."""
    out = []
    for c in range(2 ** dim):
        if all(((c >> j) & 1) == e for j, e in fixed.items()):
            out.append(c)
    return out


def resolve_sides(problem, vid):
    """Side types: a side whose corner set is shared with another patch's side is an
    interface (tag AUTO required); otherwise its tag, with AUTO meaning Dirichlet."""
    K, d = problem.num_patches, problem.dim
    keys = {}
    for k in range(K):
        for s in range(2 * d):
            j, e = divmod(s, 2)
            cs = frozenset(vid[k, c] for c in _entity_corners(d, {j: e}))
            keys.setdefault(cs, []).append((k, s))
    st = np.zeros((K, 2 * d), dtype=np.int64)
    for cs, lst in keys.items():
        if len(lst) > 2:
            raise ValueError("non-manifold side")
        for (k, s) in lst:
            tag = int(problem.side_bc[k, s])
            if len(lst) == 2:
                if tag != AUTO:
                    raise ValueError("interface side must be tagged AUTO")
                st[k, s] = INTERFACE
            else:
                st[k, s] = DIRICHLET if tag in (AUTO, DIRICHLET) else NEUMANN
    return st


def build_space(problem, level: int) -> Space:
    """Dof map, Dirichlet elimination and pieces of V_level."""
    K, d = problem.num_patches, problem.dim
    L = problem.num_levels - 1
    p = np.array(problem.degree, dtype=np.int64)
    m = np.zeros((K, d), dtype=np.int64)
    knots = []
    for k in range(K):
        row = []
        for j in range(d):
            mf = bspline.intervals_of(problem.knots[k][j], int(p[k, j]))
            if mf % (2 ** L):
                raise ValueError("finest intervals not divisible by 2^L")
            m[k, j] = mf // 2 ** (L - level)
            row.append(bspline.uniform_knots(int(m[k, j]), int(p[k, j])))
        knots.append(row)
    n = m + p
    vid = vertex_ids(np.asarray(problem.corners))
    st = resolve_sides(problem, vid)

    # canonical keys of boundary nodes -> list of (patch, local multi-index)
    occ: Dict[tuple, List[Tuple[int, tuple]]] = {}
    node_key = []
    for k in range(K):
        keys_k = {}
        grid = np.indices(tuple(n[k])).reshape(d, -1).T
        on_end = (grid == 0) | (grid == (n[k] - 1)[None, :])
        for idx in map(tuple, grid[np.any(on_end, axis=1)]):
            fixed = {}
            for j in range(d):
                if idx[j] == 0:
                    fixed[j] = 0
                elif idx[j] == n[k, j] - 1:
                    fixed[j] = 1
            ecs = _entity_corners(d, fixed)
            o = min(ecs, key=lambda c: vid[k, c])
            free = [j for j in range(d) if j not in fixed]
            pos = []
            for j in free:
                oj = (o >> j) & 1
                pos.append((vid[k, o ^ (1 << j)], idx[j] if oj == 0 else n[k, j] - 1 - idx[j]))
            pos.sort()
            key = (frozenset(vid[k, c] for c in ecs), tuple(int(q) for _, q in pos))
            keys_k[idx] = key
            occ.setdefault(key, []).append((k, idx))
        node_key.append(keys_k)

    def on_dirichlet(k, idx):
        for s in range(2 * d):
            j, e = divmod(s, 2)
            if st[k, s] == DIRICHLET and idx[j] == (0 if e == 0 else n[k, j] - 1):
                return True
        return False

    key_dir = {key: any(on_dirichlet(k, idx) for k, idx in lst) for key, lst in occ.items()}

    l2g = []
    key_id: Dict[tuple, int] = {}
    N = 0
    for k in range(K):
        new = np.ones(tuple(n[k]), dtype=bool)       # nodes that receive a fresh id here
        later = []                                   # boundary nodes numbered elsewhere
        for idx, key in node_key[k].items():
            if key_dir[key] or occ[key][0] != (k, idx):
                new[idx] = False
                if not key_dir[key]:
                    later.append((idx, key))
        ids = np.where(new, N + np.cumsum(new.ravel()).reshape(new.shape) - 1, -1)
        N += int(new.sum())
        for idx, key in node_key[k].items():
            if new[idx]:
                key_id[key] = int(ids[idx])
        for idx, key in later:
            ids[idx] = key_id[key]
        l2g.append(ids.astype(np.int64))

    space = Space(d, n, m, p, knots, l2g, N, st)

    # pieces
    owners = {}
    for key, lst in occ.items():
        owners[key] = sorted({k for k, _ in lst})
    count = np.zeros(N, dtype=np.int64)
    for k in range(K):
        drop = []
        sl = []
        for j in range(d):
            lo = st[k, 2 * j] in (INTERFACE, DIRICHLET)
            hi = st[k, 2 * j + 1] in (INTERFACE, DIRICHLET)
            drop.append((bool(lo), bool(hi)))
            sl.append(np.arange(1 if lo else 0, n[k, j] - 1 if hi else n[k, j]))
        ids = l2g[k][np.ix_(*sl)]
        if np.any(ids < 0):
            raise ValueError("patch interior contains an eliminated dof")
        space.pieces.append(Piece("interior", ids, k, tuple(range(d)), tuple(drop)))
        count[ids.ravel()] += 1
    kinds = {1: "vertex", 2: "edge", 3: "face"} if d == 3 else {1: "vertex", 2: "edge"}
    groups: Dict[frozenset, List[Tuple[tuple, int]]] = {}
    for key, lst in occ.items():
        if key_dir[key] or len(owners[key]) < 2:
            continue
        groups.setdefault(key[0], []).append((key[1], key_id[key]))
    for ecs, lst in sorted(groups.items(), key=lambda kv: min(g for _, g in kv[1])):
        ncorner = len(ecs)
        kind = kinds[{1: 1, 2: 2, 4: 3}[ncorner]]
        lst.sort()
        k0, idx0 = occ[(ecs, lst[0][0])][0]
        # piece axes in the canonical order: recover patch-local directions of k0
        fixed = {j: (0 if idx0[j] == 0 else 1) for j in range(d)
                 if idx0[j] in (0, n[k0, j] - 1)}
        free = [j for j in range(d) if j not in fixed]
        ecl = _entity_corners(d, fixed)
        o = min(ecl, key=lambda c: vid[k0, c])
        free.sort(key=lambda j: vid[k0, o ^ (1 << j)])
        if kind == "vertex":
            ids = np.array([lst[0][1]])
        else:
            shape = tuple(int(n[k0, j]) - 2 for j in free)
            ids = np.array([g for _, g in lst]).reshape(shape)
        space.pieces.append(Piece(kind, ids, k0, tuple(free)))
        count[ids.ravel()] += 1
    if not np.all(count == 1):
        raise ValueError("pieces do not partition the dofs")
    return space


def global_matrix(space: Space, patch_mats: List[sp.spmatrix]) -> sp.csr_matrix:
    """A = sum_k R_k^T A_k R_k (Sec. 4: the global matrix is the sum of the patch
    contributions), eliminated dofs dropped."""
    rows, cols, vals = [], [], []
    for k, Ak in enumerate(patch_mats):
        g = space.l2g[k].ravel()
        C = Ak.tocoo()
        r, c = g[C.row], g[C.col]
        keep = (r >= 0) & (c >= 0)
        rows.append(r[keep]); cols.append(c[keep]); vals.append(C.data[keep])
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(space.N, space.N))
    return A.tocsr()


def global_vector(space: Space, patch_vecs: List[np.ndarray]) -> np.ndarray:
    """b = sum_k R_k^T b_k."""
    b = np.zeros(space.N)
    for k, bk in enumerate(patch_vecs):
        g = space.l2g[k].ravel()
        keep = g >= 0
        np.add.at(b, g[keep], np.asarray(bk).ravel()[keep])
    return b


def stiffness(problem, space: Space, want_mass=False):
    """Global A_l (and optionally the geometry mass matrix) from the patch matrices,
    assembled element by element (patch.patch_bands)."""
    mats, masses = [], []
    for k in range(problem.num_patches):
        args = (np.asarray(problem.corners[k]), space.knots[k], space.p[k])
        mats.append(patch.bands_to_csr(patch.patch_bands(*args), space.p[k]))
        if want_mass:
            masses.append(patch.bands_to_csr(patch.patch_bands(*args, mass=True), space.p[k]))
    A = global_matrix(space, mats)
    if want_mass:
        return A, global_matrix(space, masses)
    return A


def prolongation(space_c: Space, space_f: Space) -> sp.csr_matrix:
    """Global P_l (Sec. 3): the row of a fine dof is taken from one owner patch as the
    tensor product of 1D knot-insertion matrices (the owners agree: Sec. 4, block
    triangular structure of P_l)."""
    K, d = space_f.n.shape
    P1 = [[bspline.prolongation_1d(int(space_c.m[k, j]), int(space_c.p[k, j]))
           for j in range(d)] for k in range(K)]
    done = np.zeros(space_f.N, dtype=bool)
    rows, cols, vals = [], [], []
    for k in range(K):
        Pk = sp.csr_matrix(P1[k][0])
        for j in range(1, d):
            Pk = sp.kron(Pk, sp.csr_matrix(P1[k][j]), format="csr")
        gf = space_f.l2g[k].ravel()
        gc = space_c.l2g[k].ravel()
        sel = np.nonzero(gf >= 0)[0]
        sel = sel[~done[gf[sel]]]
        done[gf[sel]] = True
        C = Pk[sel].tocoo()
        keep = (gc[C.col] >= 0) & (C.data != 0)
        rows.append(gf[sel][C.row[keep]]); cols.append(gc[C.col[keep]]); vals.append(C.data[keep])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(space_f.N, space_c.N))
