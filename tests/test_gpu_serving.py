"""Serving layer (igamg_server_*): requests of several models (2D and 3D, different
sizes) submitted together and answered by concurrent workers.

  * each answer is bit-identical to solving that request alone through igamg_solve
    (the served solve is the single-problem path on a resident hierarchy), also for the
    requests of a 2D rectangle-patch model that a worker takes together and solves with
    igamg_solve_multi (forced FD engine); with the autotuned default such grouped answers
    equal the single solves to rounding;
  * with a device-memory budget that holds one hierarchy at a time, hierarchies are
    evicted and rebuilt and the answers are unchanged;
  * a model larger than the budget is answered with IGAMG_ERR_OOM, the others are served;
  * latency bookkeeping is ordered (submit <= start <= done)."""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def models():
    return [workloads.rect_grid_2d(2, 3, 16), workloads.perturbed_grid_2d(2, 4, 16, 5, 4),
            workloads.perturbed_cube_3d(2, 2, 4, 3, 3), workloads.rect_grid_2d(3, 2, 32),
            workloads.perturbed_cube_3d(2, 2, 12, 3, 3)]


def fma_options():
    from paper_1804_02539_gb300 import igamg
    o = igamg.igamg_default_options()
    o.fd_engine = 1
    return o


def alone(pr, b, opts=None):
    from paper_1804_02539_gb300 import igamg
    c = igamg.Context(pr, opts)
    x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    res, st = c.solve(torch.tensor(b, device="cuda"), x, 1e-8)
    out = x.cpu().numpy()
    c.free()
    return out, res.iters


def similar_models():
    return [workloads.rect_grid_2d(2, p, 32) for p in range(2, 7)]


def estimates(mods):
    from paper_1804_02539_gb300 import igamg
    srv = igamg.Server(workers=1)
    est = [srv.add_model(pr)[2] for pr in mods]
    srv.free()
    return est


def serve(budget, reqs, workers=3, mods=None, opts=None):
    from paper_1804_02539_gb300 import igamg
    mods = mods or models()
    srv = igamg.Server(opts, workers=workers, hbm_budget_bytes=budget)
    ids = [srv.add_model(pr) for pr in mods]
    sub = []
    for m, seed in reqs:
        b = np.random.default_rng(seed).uniform(-1, 1, ids[m][1])
        rid, x = srv.submit(ids[m][0], b, 1e-8)
        sub.append((m, b, rid, x))
    out = [(m, b, x, srv.wait(rid)) for m, b, rid, x in sub]
    stats = srv.stats()
    srv.free()
    return out, stats


REQS = [(i % 5, 100 + i) for i in range(15)]


def test_served_answers_match_single_solves():
    out, stats = serve(8 << 30, REQS, opts=fma_options())
    assert stats["completed"] == len(REQS) and stats["setups"] == 5 and stats["evictions"] == 0
    assert stats["groups"] > 0 and stats["grouped"] == sum(1 for *_, i in out if i["group"] > 1)
    prs = models()
    for m, b, x, info in out:
        ref, its = alone(prs[m], b, fma_options())
        assert info["status"] == 0 and info["iters"] == its
        assert np.array_equal(x, ref)
        assert info["t_submit_ms"] <= info["t_start_ms"] <= info["t_done_ms"]


def test_grouped_requests_autotuned():
    """Twelve requests of one 2D rectangle-patch model and four of a 3D model submitted at
    once to one worker: the 2D ones are answered in groups (at most 16), the 3D ones one at a
    time; every answer meets the tolerance and equals the request solved alone to rounding."""
    mods = [workloads.rect_grid_2d(3, 3, 32), workloads.perturbed_cube_3d(2, 2, 4, 3, 3)]
    reqs = [(0, 700 + i) for i in range(12)] + [(1, 800 + i) for i in range(4)]
    out, stats = serve(8 << 30, reqs, workers=1, mods=mods)
    assert stats["completed"] == len(reqs) and stats["groups"] >= 1
    for m, b, x, info in out:
        assert info["status"] == 0 and info["relres"] <= 1e-8
        assert info["t_submit_ms"] <= info["t_start_ms"] <= info["t_done_ms"]
        if m == 1:
            assert info["group"] == 1
        ref, its = alone(mods[m], b)
        assert abs(info["iters"] - its) <= 1
        assert np.linalg.norm(x - ref) <= (1e-8 if info["iters"] == its else 1e-6) * np.linalg.norm(ref)
    assert max(info["group"] for m, *_, info in out if m == 0) > 1


def test_eviction_under_a_small_budget():
    """Five hierarchies of similar size; the budget holds the largest estimate, which is
    less than all five together: every hierarchy is evicted and rebuilt at least once."""
    mods = similar_models()
    est = estimates(mods)
    out, full = serve(8 << 30, REQS[:5], mods=mods, opts=fma_options())
    assert full["device_bytes"] > 1.1 * max(est)   # all five do not fit the budget below
    out, stats = serve(int(1.05 * max(est)), REQS, workers=2, mods=mods, opts=fma_options())
    assert stats["evictions"] > 0 and stats["completed"] == len(REQS)
    for m, b, x, info in out:
        ref, _ = alone(mods[m], b, fma_options())
        assert info["status"] == 0 and np.array_equal(x, ref)


def test_model_larger_than_budget_is_refused():
    est = estimates(models())
    assert est[4] > est[0]
    out, stats = serve((est[0] + est[4]) // 2, [(0, 1), (4, 2), (0, 3)], workers=1)
    statuses = [info["status"] for _, _, _, info in out]
    assert statuses == [0, 4, 0]  # IGAMG_ERR_OOM for the model that never fits


def test_bad_requests_are_rejected():
    from paper_1804_02539_gb300 import igamg
    srv = igamg.Server(workers=1, hbm_budget_bytes=1 << 30)
    m, n, _ = srv.add_model(workloads.unit_square_quadrants(8, 2, 4))
    with pytest.raises(igamg.IgamgError):
        srv.submit(m + 1, np.zeros(n))             # unknown model
    with pytest.raises(igamg.IgamgError):
        srv.wait(12345)                            # unknown request
    bad = workloads.unit_square_quadrants(6, 2, 4)  # 6 intervals cannot make 4 levels
    with pytest.raises(igamg.IgamgError):
        srv.add_model(bad)
    rid, x = srv.submit(m, np.zeros(n))            # zero load: zero answer, no iterations
    info = srv.wait(rid)
    assert info["status"] == 0 and info["iters"] == 0 and not x.any()
    srv.free()
