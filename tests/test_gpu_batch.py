"""Batched solves of independent problems (uneven sizes, degrees, patch counts, 2D and
3D, rectangle and bilinear patches) through igamg_setup_batch / igamg_solve_batch:

  * every batch result is bit-identical to the same problem solved alone, whatever the
    number of workers (the batch only schedules the single-problem path);
  * sampled members agree with the oracle's direct solve of the same linear system;
  * a failing problem is reported by index and leaves nothing allocated."""
import numpy as np
import pytest

import workloads
from oracle import solver
from tests.helpers import permutation, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def mixed_batch():
    probs = workloads.batch_problems(10, seed=11, m_choices=(8, 16), K_choices=(4, 9))
    probs.append(workloads.perturbed_grid_2d(2, 3, 16, 5, 4))    # bilinear patches, mixed BCs
    probs.append(workloads.perturbed_cube_3d(2, 2, 4, 3, 3))     # 3D
    probs.append(workloads.unit_square_quadrants(8, 2, 4))       # the smallest case
    return probs


@pytest.fixture(scope="module")
def batch():
    from paper_1804_02539_gb300 import igamg
    probs = mixed_batch()
    b = igamg.Batch(probs, workers=4)
    rhs = [torch.tensor(workloads.rhs_coefficients(c.num_dofs(), 100 + i), device="cuda")
           for i, c in enumerate(b.contexts)]
    yield probs, b, rhs
    b.free()


def test_batch_matches_single_solves(batch):
    from paper_1804_02539_gb300 import igamg
    probs, b, rhs = batch
    xs = [torch.zeros_like(r) for r in rhs]
    st, res, sts = b.solve(rhs, xs, 1e-8)
    assert st == 0 and all(s == 0 for s in sts)
    for i, pr in enumerate(probs):
        c = igamg.Context(pr)
        x = torch.zeros_like(rhs[i])
        r1, _ = c.solve(rhs[i], x, 1e-8)
        assert r1.iters == res[i].iters, i
        assert torch.equal(x, xs[i]), i
        assert res[i].relres <= 1e-8
        c.free()


def test_worker_count_does_not_change_results(batch):
    from paper_1804_02539_gb300 import igamg
    probs, b, rhs = batch
    x4 = [torch.zeros_like(r) for r in rhs]
    b.solve(rhs, x4, 1e-8)
    b1 = igamg.Batch(probs, workers=1)
    x1 = [torch.zeros_like(r) for r in rhs]
    st, res, sts = b1.solve(rhs, x1, 1e-8)
    assert st == 0
    for a, c in zip(x4, x1):
        assert torch.equal(a, c)
    b1.free()


def test_batch_members_match_oracle_direct_solve(batch):
    probs, b, rhs = batch
    xs = [torch.zeros_like(r) for r in rhs]
    b.solve(rhs, xs, 1e-10)
    for i in (0, 5, len(probs) - 3, len(probs) - 2, len(probs) - 1):
        pr = probs[i]
        H = solver.build_hierarchy(pr)
        sp = H.levels[-1].space
        perm = permutation(sp, b.contexts[i].dof_map())
        bl = rhs[i].cpu().numpy()[perm]
        ref = solver.direct_solve(H.levels[-1].A, bl)
        assert rel(xs[i].cpu().numpy()[perm], ref) < 1e-7, i


def test_repeated_batch_solves_and_initial_guess(batch):
    """A second solve started at the first one's answer stays on it (the initial guess is
    used, the resident hierarchies are reused)."""
    probs, b, rhs = batch
    xs = [torch.zeros_like(r) for r in rhs]
    b.solve(rhs, xs, 1e-10)
    x2 = [x.clone() for x in xs]
    st, res, _ = b.solve(rhs, x2, 1e-4)
    assert st == 0
    for a, c in zip(xs, x2):
        assert rel(c.cpu().numpy(), a.cpu().numpy()) < 1e-9


def test_batch_reports_failing_problem():
    from paper_1804_02539_gb300 import igamg
    good = workloads.unit_square_quadrants(8, 2, 4)
    bad = workloads.unit_square_quadrants(8, 2, 4)
    bad.num_levels = 9          # more levels than 8 intervals allow
    with pytest.raises(igamg.IgamgError) as e:
        igamg.Batch([good, good, bad, good], workers=2)
    assert "problem 2" in str(e.value)


def test_batch_of_one_and_more_workers_than_problems():
    from paper_1804_02539_gb300 import igamg
    pr = workloads.unit_square_quadrants(8, 2, 4)
    b = igamg.Batch([pr], workers=8)
    rhs = [torch.tensor(workloads.rhs_coefficients(b.contexts[0].num_dofs(), 1), device="cuda")]
    xs = [torch.zeros_like(rhs[0])]
    st, res, sts = b.solve(rhs, xs, 1e-8)
    c = igamg.Context(pr)
    x = torch.zeros_like(rhs[0])
    c.solve(rhs[0], x, 1e-8)
    assert st == 0 and torch.equal(x, xs[0])
    c.free()
    b.free()
