"""Parity of the tensor-core fast-diagonalisation path at sizes where it runs its MMAs
(Sec. 3: the patch-interior smoother in diagonalised form and the face smoothers of
Eq. additive; Algorithm 1; PCG of Sec. 4), against the FP64 oracle.

The cases have interiors and faces wider than 32 in every direction, so every product of
the tensor-core FD (2D: four products per interior; 3D: six "contract the leading mode"
stages per interior, four per face) has tiles with more than 32 valid rows and columns:
  * 2D, 2x2 patches, p=3, 32 intervals: interiors of 33 x 33 .. 34 x 34, so the smallest
    has exactly 33 valid rows; full hierarchy;
  * 3D, one patch, p=2, 32 intervals, Neumann on the +x, +y, +z sides: interior 33^3;
    full hierarchy: smoother on every level, one cycle, PCG iterates after k iterations,
    iteration counts, tight solve;
  * 3D, 2x2x2 patches, p=3, 32 intervals: interiors 33^3, faces 33 x 33, edges of 33; the
    finest smoother against the oracle's local smoothers (no assembly needed).
Each runs with the tensor cores forced on every level (fd_engine = 2) and with the
autotuned default.  Tolerances as in the other parity tests: smoother 1e-12, one cycle
1e-11, PCG iterates 1e-10, counts +-1."""
import numpy as np
import pytest

import workloads
from oracle import multipatch, smoother, solver
from tests.helpers import permutation, rel, to_lib, from_lib

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def grid2d_p3_m32():
    return workloads.perturbed_grid_2d(2, 3, 32, 4, 5)


def cube1_p2_m32_neumann():
    pr = workloads.perturbed_cube_3d(1, 2, 32, 3, 5)
    pr.side_bc[0, [1, 3, 5]] = workloads.SIDE_NEUMANN
    return pr


def cube2_p3_m32():
    return workloads.perturbed_cube_3d(2, 3, 32, 3, 3)


FULL = {"grid2d_p3_m32": grid2d_p3_m32, "cube1_p2_m32_neumann": cube1_p2_m32_neumann}
_CACHE = {}


def dev(v):
    return torch.tensor(np.ascontiguousarray(v), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def setup_full(name):
    """Oracle hierarchy, the autotuned context and a context with the tensor cores forced."""
    if name not in _CACHE:
        from paper_1804_02539_gb300 import igamg
        pr = FULL[name]()
        H = solver.build_hierarchy(pr)
        o = igamg.igamg_default_options()
        o.fd_engine = 2
        ctxs = {"auto": igamg.Context(pr), "tc": igamg.Context(pr, o)}
        perms = [permutation(H.levels[l].space, ctxs["auto"].dof_map(l)) for l in range(pr.num_levels)]
        _CACHE[name] = (pr, H, ctxs, perms)
    return _CACHE[name]


def test_cases_are_wider_than_32():
    """The cases reach the MMA tiles: every interior (and face) of the finest level has more
    than 32 dofs per direction, and the smallest 2D interior has exactly 33."""
    for make in (grid2d_p3_m32, cube1_p2_m32_neumann, cube2_p3_m32):
        pr = make()
        sp_ = multipatch.build_space(pr, pr.num_levels - 1)
        shapes = [pc.ids.shape for pc in sp_.pieces if pc.kind in ("interior", "face")]
        assert shapes and min(min(s) for s in shapes) >= 33
    sp_ = multipatch.build_space(grid2d_p3_m32(), 3)
    assert min(min(pc.ids.shape) for pc in sp_.pieces if pc.kind == "interior") == 33


@pytest.mark.parametrize("eng", ["tc", "auto"])
@pytest.mark.parametrize("name", list(FULL))
def test_smoother_every_level(name, eng):
    pr, H, ctxs, perms = setup_full(name)
    rng = np.random.default_rng(1)
    for l in range(1, pr.num_levels):
        r = rng.normal(size=H.levels[l].space.N)
        z = torch.empty_like(dev(r))
        ctxs[eng].smooth(l, dev(to_lib(perms[l], r)), z)
        ref = smoother.apply_smoother(H.levels[l].smooth, r)
        assert rel(from_lib(perms[l], host(z)), ref) < 1e-12, l


@pytest.mark.parametrize("eng", ["tc", "auto"])
@pytest.mark.parametrize("name", list(FULL))
def test_one_cycle(name, eng):
    pr, H, ctxs, perms = setup_full(name)
    r = np.random.default_rng(4).normal(size=H.levels[-1].space.N)
    z = torch.empty_like(dev(r))
    ctxs[eng].precondition(dev(to_lib(perms[-1], r)), z)
    assert rel(from_lib(perms[-1], host(z)), solver.precondition(H, r)) < 1e-11


@pytest.mark.parametrize("eng", ["tc", "auto"])
@pytest.mark.parametrize("name", list(FULL))
def test_pcg_parity(name, eng):
    from paper_1804_02539_gb300 import igamg
    pr, H, ctxs, perms = setup_full(name)
    N = H.levels[-1].space.N
    b = workloads.rhs_coefficients(N, 5)
    ref = solver.pcg(H, b, tol=1e-8)
    x = torch.zeros(N, dtype=torch.float64, device="cuda")
    res, st = ctxs[eng].solve(dev(to_lib(perms[-1], b)), x, 1e-8)
    assert st == igamg.IGAMG_OK
    assert abs(res.iters - ref.iters) <= 1, (res.iters, ref.iters)
    k = ref.iters
    fixed = solver.pcg(H, b, fixed_iters=k)
    o = igamg.igamg_default_options()
    o.max_iter = k
    if eng == "tc":
        o.fd_engine = 2
    ck = igamg.Context(pr, o)
    xk = torch.zeros_like(x)
    rk, _ = ck.solve(dev(to_lib(perms[-1], b)), xk, 0.0)
    assert rk.iters == k
    assert rel(from_lib(perms[-1], host(xk)), fixed.x) < 1e-10
    ck.free()
    tight = solver.pcg(H, b, tol=1e-13, max_iter=300)
    xt = torch.zeros_like(x)
    ctxs[eng].solve(dev(to_lib(perms[-1], b)), xt, 1e-13)
    assert rel(from_lib(perms[-1], host(xt)), tight.x) < 1e-10


@pytest.mark.parametrize("eng", [2, 0])
def test_cube2x2x2_finest_smoother(eng):
    """2x2x2 patches at 33 dofs per interior direction: interiors (six mode-product
    stages), faces (2D FD of 33 x 33), edges and the vertex, every piece against the
    oracle's local smoother."""
    from paper_1804_02539_gb300 import igamg
    pr = cube2_p3_m32()
    L = pr.num_levels - 1
    sp_ = multipatch.build_space(pr, L)
    sms = smoother.build_smoother(sp_, L)
    o = igamg.igamg_default_options()
    o.fd_engine = eng
    ctx = igamg.Context(pr, o)
    perm = permutation(sp_, ctx.dof_map(L))
    r = np.random.default_rng(7).normal(size=sp_.N)
    z = torch.empty(sp_.N, dtype=torch.float64, device="cuda")
    ctx.smooth(L, dev(to_lib(perm, r)), z)
    got = from_lib(perm, host(z))
    kinds = set()
    for s in sms:
        ids = s.piece.ids
        ref = s.Dinv * r[ids] if s.piece.kind == "vertex" else smoother.fd_apply(s.Us, s.Dinv, r[ids])
        assert np.linalg.norm(got[ids] - ref) <= 1e-12 * np.linalg.norm(ref), s.piece.kind
        kinds.add(s.piece.kind)
    assert kinds == {"interior", "face", "edge", "vertex"}
    assert rel(got, smoother.apply_smoother(sms, r)) < 1e-12
    ctx.free()
