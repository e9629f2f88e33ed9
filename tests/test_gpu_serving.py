"""Serving layer (igamg_server_*): requests of several models (2D and 3D, different
sizes) submitted together and answered by concurrent workers.

  * each answer is bit-identical to solving that request alone through igamg_solve
    (the served solve is the single-problem path on a resident hierarchy);
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


def alone(pr, b):
    from paper_1804_02539_gb300 import igamg
    c = igamg.Context(pr)
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


def serve(budget, reqs, workers=3, mods=None):
    from paper_1804_02539_gb300 import igamg
    mods = mods or models()
    srv = igamg.Server(workers=workers, hbm_budget_bytes=budget)
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
    out, stats = serve(8 << 30, REQS)
    assert stats["completed"] == len(REQS) and stats["setups"] == 5 and stats["evictions"] == 0
    prs = models()
    for m, b, x, info in out:
        ref, its = alone(prs[m], b)
        assert info["status"] == 0 and info["iters"] == its
        assert np.array_equal(x, ref)
        assert info["t_submit_ms"] <= info["t_start_ms"] <= info["t_done_ms"]


def test_eviction_under_a_small_budget():
    """Five hierarchies of similar size; the budget holds the largest estimate, which is
    less than all five together: every hierarchy is evicted and rebuilt at least once."""
    mods = similar_models()
    est = estimates(mods)
    out, full = serve(8 << 30, REQS[:5], mods=mods)
    assert full["device_bytes"] > 1.1 * max(est)   # all five do not fit the budget below
    out, stats = serve(int(1.05 * max(est)), REQS, workers=2, mods=mods)
    assert stats["evictions"] > 0 and stats["completed"] == len(REQS)
    for m, b, x, info in out:
        ref, _ = alone(mods[m], b)
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
