"""Parity at the benchmark size (2D, K=16, p=4, 256 intervals per patch direction,
1,073,296 dofs, the configuration bench.py times): sampled outputs the oracle computes
one by one, and properties that hold at any size.

  * stiffness apply: rows of A_L for sampled dofs (interior, interface, Neumann-boundary
    and vertex dofs) assembled by the oracle from the Gauss points of their support only;
  * smoother: the patch-interior fast-diagonalisation block of one patch and the edge
    and vertex blocks, recomputed by the oracle for those pieces;
  * preconditioner symmetry <B x, y> = <x, B y> (Sec. 3: same smoother pre and post);
  * the PCG solve converges to 1e-8 within the iteration band of the oracle at smaller
    sizes, and the residual recomputed on sampled rows by the oracle is consistent."""
import numpy as np
import pytest

import workloads
from oracle import multipatch, patch, smoother
from tests.helpers import permutation

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def big():
    from paper_1804_02539_gb300 import igamg
    pr = workloads.CONFIGS["grid2d_K16_p4_m256"]()
    ctx = igamg.Context(pr)
    space = multipatch.build_space(pr, pr.num_levels - 1)
    perm = permutation(space, ctx.dof_map())
    return pr, ctx, space, perm


def oracle_rows(pr, space, gids):
    """Rows of the global A for the given oracle dof ids: sum over owner patches of the
    patch rows, each from the Gauss points of that dof's support only."""
    rows = {}
    p = int(space.p[0, 0])
    for g in gids:
        acc = {}
        for k in range(pr.num_patches):
            where = np.argwhere(space.l2g[k] == g)
            if len(where) == 0:
                continue
            i = where[0]
            win = [(max(int(i[j]) - p, 0), min(int(i[j]) + 1, int(space.m[k, j]))) for j in range(space.dim)]
            A = patch.patch_matrices(np.asarray(pr.corners[k]), space.knots[k], space.p[k], elem_window=win)
            li = int(np.ravel_multi_index(tuple(i), tuple(space.n[k])))
            row = A.getrow(li).tocoo()
            gl = space.l2g[k].ravel()[row.col]
            for c, v in zip(gl, row.data):
                if c >= 0:
                    acc[c] = acc.get(c, 0.0) + v
        rows[g] = acc
    return rows


def sample_dofs(space, rng, count=40, neumann_patch=15):
    """`count` random dofs, the middle dof of every face, edge and vertex piece, and (2D)
    the last dof of patch `neumann_patch`'s interior (a corner on Neumann sides)."""
    N = space.N
    picks = list(rng.choice(N, count, replace=False))
    for pc in space.pieces:              # at least one dof of every piece kind
        if pc.kind in ("face", "edge", "vertex"):
            picks.append(int(pc.ids.ravel()[len(pc.ids.ravel()) // 2]))
    if neumann_patch is not None:
        picks.append(int(space.pieces[neumann_patch].ids[-1, -1]))
    return sorted(set(int(x) for x in picks))


def test_apply_sampled_rows(big):
    pr, ctx, space, perm = big
    rng = np.random.default_rng(0)
    x = rng.normal(size=space.N)
    xl = np.empty_like(x)
    xl[perm] = x
    y = torch.empty(space.N, dtype=torch.float64, device="cuda")
    ctx.apply(-1, torch.tensor(xl, device="cuda"), y)
    yl = y.cpu().numpy()[perm]
    gids = sample_dofs(space, rng)
    rows = oracle_rows(pr, space, gids)
    for g in gids:
        cols = np.array(list(rows[g].keys()))
        vals = np.array(list(rows[g].values()))
        ref = vals @ x[cols]
        scale = np.abs(vals) @ np.abs(x[cols])
        assert abs(yl[g] - ref) <= 1e-13 * scale, (g, yl[g], ref)


def test_smoother_sampled_pieces(big):
    pr, ctx, space, perm = big
    rng = np.random.default_rng(1)
    r = rng.normal(size=space.N)
    rl = np.empty_like(r)
    rl[perm] = r
    z = torch.empty(space.N, dtype=torch.float64, device="cuda")
    ctx.smooth(pr.num_levels - 1, torch.tensor(rl, device="cuda"), z)
    zl = z.cpu().numpy()[perm]
    sms = smoother.build_smoother(space, pr.num_levels - 1)
    chosen = [sms[i] for i in (0, 5, 15)] + [s for s in sms if s.piece.kind != "interior"][::5]
    for s in chosen:
        ids = s.piece.ids
        if s.piece.kind == "vertex":
            ref = s.Dinv * r[ids]
        else:
            ref = smoother.fd_apply(s.Us, s.Dinv, r[ids])
        got = zl[ids]
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref), s.piece.kind


def test_preconditioner_symmetric(big):
    pr, ctx, space, perm = big
    rng = np.random.default_rng(2)
    x = torch.tensor(rng.normal(size=space.N), device="cuda")
    y = torch.tensor(rng.normal(size=space.N), device="cuda")
    bx, by = torch.empty_like(x), torch.empty_like(y)
    ctx.precondition(x, bx)
    ctx.precondition(y, by)
    a, b = float(torch.dot(bx, y)), float(torch.dot(x, by))
    assert abs(a - b) <= 1e-12 * abs(a)
    assert float(torch.dot(bx, x)) > 0


def test_solve_converges_and_sampled_residual(big):
    pr, ctx, space, perm = big
    N = space.N
    coef = torch.tensor(workloads.rhs_coefficients(N, 2), device="cuda")
    b = torch.empty(N, dtype=torch.float64, device="cuda")
    ctx.rhs_from_coefs(coef, b)
    x = torch.zeros(N, dtype=torch.float64, device="cuda")
    res, st = ctx.solve(b, x, 1e-8)
    assert st == 0 and res.relres <= 1e-8
    assert 20 <= res.iters <= 40          # oracle: 27-28 at 16..64 intervals (h-robust)
    bl, xl = b.cpu().numpy()[perm], x.cpu().numpy()[perm]
    rng = np.random.default_rng(3)
    gids = sample_dofs(space, rng, 20)
    rows = oracle_rows(pr, space, gids)
    bnorm = np.linalg.norm(bl)
    for g in gids:
        cols = np.array(list(rows[g].keys()))
        vals = np.array(list(rows[g].values()))
        # every single residual entry is bounded by the residual norm
        assert abs(bl[g] - vals @ xl[cols]) <= 1.01e-8 * bnorm
