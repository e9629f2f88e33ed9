"""The lockstep batch engine: PCG for many independent 2D rectangle-patch problems at once,
every step of Algorithm 1 (apply, smoother pieces, transfers, coarse solves) one launch over
all problems at the same depth below their finest level, one graph replay per PCG
iteration of the whole batch.

  * the engine is chosen for such batches (and the worker-stream engine otherwise);
  * with a forced FD engine (FMA GEMMs, tensor cores, one-block kernels, row blocks) every
    answer and iteration count is bit-identical to the same problem solved alone, so
    problems that converge early keep their iterate; with the autotuned default the
    lockstep engine puts every level whose tensor-core stages exist on the tensor cores
    (a problem timed alone may have picked FMA GEMMs), which changes results by rounding
    only (1e-9 relative, iteration counts +-1);
  * sampled members agree with the oracle's direct solve of the same linear system;
  * a second solve from the first one's answer stays on it (initial guess, reuse)."""
import numpy as np
import pytest

import workloads
from oracle import solver
from tests.helpers import permutation, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rect_batch():
    probs = workloads.batch_problems(14, seed=12, m_choices=(8, 16, 32, 64), K_choices=(4, 9, 16))
    probs.append(workloads.unit_square_quadrants(8, 2, 4))
    return probs


def _rhs(b, seed0):
    return [torch.tensor(workloads.rhs_coefficients(c.num_dofs(), seed0 + i), device="cuda")
            for i, c in enumerate(b.contexts)]


@pytest.mark.parametrize("fd_engine", [1, 2, 3, 4])
def test_lockstep_matches_single_solves(fd_engine):
    from paper_1804_02539_gb300 import igamg
    probs = rect_batch()
    o = igamg.igamg_default_options()
    o.fd_engine = fd_engine
    b = igamg.Batch(probs, o)
    assert b.engine() == "lockstep"
    rhs = _rhs(b, 200)
    xs = [torch.zeros_like(r) for r in rhs]
    st, res, sts = b.solve(rhs, xs, 1e-8)
    assert st == 0 and all(s == 0 for s in sts)
    its = set()
    for i, pr in enumerate(probs):
        c = igamg.Context(pr, o)
        x = torch.zeros_like(rhs[i])
        r1, _ = c.solve(rhs[i], x, 1e-8)
        assert r1.iters == res[i].iters, (i, r1.iters, res[i].iters)
        assert torch.equal(x, xs[i]), i
        assert res[i].relres <= 1e-8
        its.add(r1.iters)
        c.free()
    assert len(its) > 1     # members stop at different iterations: the masking is exercised
    b.free()


def test_lockstep_autotuned_matches_single_solves_to_rounding():
    from paper_1804_02539_gb300 import igamg
    probs = rect_batch()
    b = igamg.Batch(probs)
    rhs = _rhs(b, 400)
    xs = [torch.zeros_like(r) for r in rhs]
    st, res, sts = b.solve(rhs, xs, 1e-8)
    assert st == 0
    stats = b.stats()
    assert stats["launches"] > 0 and stats["flops"] > 0
    for i, pr in enumerate(probs):
        c = igamg.Context(pr)
        x = torch.zeros_like(rhs[i])
        r1, _ = c.solve(rhs[i], x, 1e-8)
        assert abs(r1.iters - res[i].iters) <= 1, i
        # the same iterate up to the FD rounding; one iteration apart at most the tolerance
        assert rel(xs[i].cpu().numpy(), x.cpu().numpy()) < (1e-9 if r1.iters == res[i].iters else 1e-6), i
        c.free()
    b.free()


def test_lockstep_equals_worker_streams_and_oracle():
    from paper_1804_02539_gb300 import igamg
    probs = rect_batch()
    o = igamg.igamg_default_options()
    o.fd_engine = 2
    b = igamg.Batch(probs, o)
    o.batch_engine = 1
    bs = igamg.Batch(probs, o, workers=4)
    assert b.engine() == "lockstep" and bs.engine() == "streams"
    rhs = _rhs(b, 300)
    x1 = [torch.zeros_like(r) for r in rhs]
    x2 = [torch.zeros_like(r) for r in rhs]
    b.solve(rhs, x1, 1e-10)
    bs.solve(rhs, x2, 1e-10)
    for a, c in zip(x1, x2):
        assert torch.equal(a, c)
    for i in (0, 3, len(probs) - 1):
        H = solver.build_hierarchy(probs[i])
        sp = H.levels[-1].space
        perm = permutation(sp, b.contexts[i].dof_map())
        ref = solver.direct_solve(H.levels[-1].A, rhs[i].cpu().numpy()[perm])
        assert rel(x1[i].cpu().numpy()[perm], ref) < 1e-7, i
    # a second solve from the answer stays on it
    x3 = [x.clone() for x in x1]
    st, res, _ = b.solve(rhs, x3, 1e-4)
    assert st == 0
    for a, c in zip(x1, x3):
        assert rel(c.cpu().numpy(), a.cpu().numpy()) < 1e-9
    b.free()
    bs.free()


def test_outside_scope_uses_worker_streams():
    from paper_1804_02539_gb300 import igamg
    probs = [workloads.perturbed_grid_2d(2, 3, 16, 5, 4), workloads.unit_square_quadrants(8, 2, 4)]
    b = igamg.Batch(probs)
    assert b.engine() == "streams"      # bilinear (non-rectangle) patches
    b.free()


# ---------------------------------------------------------------- several right-hand sides

def _multi_rhs(ctx, count, seed0):
    n = ctx.num_dofs()
    return [torch.tensor(workloads.rhs_coefficients(n, seed0 + i), device="cuda") for i in range(count)]


@pytest.mark.parametrize("fd_engine", [1, 2])
def test_solve_multi_matches_single_solves(fd_engine):
    """igamg_solve_multi on one context (its work arrays copied per extra right-hand side,
    the constant arrays shared): every answer and iteration count bit-identical to the same
    right-hand side solved alone, also after a call with more right-hand sides (engines kept
    per count, copies reused)."""
    from paper_1804_02539_gb300 import igamg
    o = igamg.igamg_default_options()
    o.fd_engine = fd_engine
    c = igamg.Context(workloads.rect_grid_2d(3, 3, 32), o)
    for count, seed in ((5, 10), (3, 40), (5, 70)):
        rhs = _multi_rhs(c, count, seed)
        if count == 3:
            rhs[1] = rhs[1] * 1e-3          # a different scale: stops at another iteration
        xs = [torch.zeros_like(r) for r in rhs]
        st, res, sts = c.solve_multi(rhs, xs, 1e-9)
        assert st == 0 and all(s == 0 for s in sts)
        for i, r in enumerate(rhs):
            x = torch.zeros_like(r)
            r1, _ = c.solve(r, x, 1e-9)
            assert r1.iters == res[i].iters and torch.equal(x, xs[i]), (count, i)
            assert res[i].relres <= 1e-9
    c.free()


def test_solve_multi_autotuned_and_oracle():
    """The autotuned default (the lockstep engine may put levels on the tensor cores that a
    single solve ran on FMA GEMMs): answers equal single solves to rounding and the oracle's
    direct solve of the same system."""
    from paper_1804_02539_gb300 import igamg
    pr = workloads.rect_grid_2d(2, 4, 64)
    c = igamg.Context(pr)
    rhs = _multi_rhs(c, 6, 100)
    xs = [torch.zeros_like(r) for r in rhs]
    st, res, _ = c.solve_multi(rhs, xs, 1e-10)
    assert st == 0
    for i, r in enumerate(rhs):
        x = torch.zeros_like(r)
        r1, _ = c.solve(r, x, 1e-10)
        assert abs(r1.iters - res[i].iters) <= 1
        assert rel(xs[i].cpu().numpy(), x.cpu().numpy()) < 1e-8, i
    H = solver.build_hierarchy(pr)
    sp = H.levels[-1].space
    perm = permutation(sp, c.dof_map())
    for i in (0, 5):
        ref = solver.direct_solve(H.levels[-1].A, rhs[i].cpu().numpy()[perm])
        assert rel(xs[i].cpu().numpy()[perm], ref) < 1e-8, i
    c.free()


def test_solve_multi_precision_variant_runs_fp64():
    """A BF16-variant context: the right-hand sides run the FP64 lockstep numerics and meet
    the tolerance; the answers agree with the context's own mixed-precision solves to the
    tolerance's level."""
    from paper_1804_02539_gb300 import igamg
    o = igamg.igamg_default_options()
    o.precision = igamg.IGAMG_BF16
    c = igamg.Context(workloads.rect_grid_2d(3, 4, 32), o)
    rhs = _multi_rhs(c, 4, 300)
    xs = [torch.zeros_like(r) for r in rhs]
    st, res, _ = c.solve_multi(rhs, xs, 1e-8)
    assert st == 0 and all(r.relres <= 1e-8 for r in res)
    for i, r in enumerate(rhs):
        x = torch.zeros_like(r)
        c.solve(r, x, 1e-8)
        assert rel(xs[i].cpu().numpy(), x.cpu().numpy()) < 1e-6, i
    c.free()


def test_solve_multi_outside_scope_solves_one_by_one():
    """A 3D problem (outside the lockstep scope): the right-hand sides are solved one after
    the other, bit-identical to igamg_solve."""
    from paper_1804_02539_gb300 import igamg
    c = igamg.Context(workloads.perturbed_cube_3d(2, 2, 4, 3, 3))
    rhs = _multi_rhs(c, 3, 500)
    xs = [torch.zeros_like(r) for r in rhs]
    st, res, _ = c.solve_multi(rhs, xs, 1e-8)
    assert st == 0
    for i, r in enumerate(rhs):
        x = torch.zeros_like(r)
        r1, _ = c.solve(r, x, 1e-8)
        assert r1.iters == res[i].iters and torch.equal(x, xs[i])
    c.free()
