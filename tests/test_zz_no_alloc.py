"""igamg_fd_apply_noalloc: the fast-diagonalisation apply for callers that cannot allocate
device memory (a host framework that owns the allocator, a fixed-budget or real-time
caller, ...).  It must give the same result as igamg_fd_apply, which takes caller-provided
scratch, on consecutive calls that share its built-in scratch array, and must reject tiles
beyond its fixed limit.  Kept in its own file, collected last."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-13   # relative 2-norm, the FP64 tolerance used for the FD contraction elsewhere


def _lib():
    from paper_1804_02539_gb300 import igamg
    return igamg.lib()


def _tile(seed, n0, n1, ld_pad):
    rng = np.random.default_rng(seed)
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    U0, U1 = dev(rng.normal(size=(n0, n0))), dev(rng.normal(size=(n1, n1)))
    Dinv = dev(rng.uniform(0.1, 1.0, size=(n0, n1)))
    R = dev(rng.normal(size=(n0, n1 + ld_pad)))
    return U0, U1, Dinv, R


def _with_scratch(U0, U1, Dinv, R, n1, tau):
    n0 = U0.shape[0]
    Z = torch.zeros((n0, n1), dtype=torch.float64, device="cuda")
    scratch = torch.empty(2 * n0 * n1, dtype=torch.float64, device="cuda")
    st = _lib().igamg_fd_apply(n0, n1, C.c_void_p(U0.data_ptr()), C.c_void_p(U1.data_ptr()),
                               C.c_void_p(Dinv.data_ptr()), C.c_void_p(R.data_ptr()), R.stride(0), tau,
                               C.c_void_p(Z.data_ptr()), n1, C.c_void_p(scratch.data_ptr()), None)
    assert st == 0
    return Z


def _no_alloc(U0, U1, Dinv, R, n1, tau):
    n0 = U0.shape[0]
    Z = torch.full((n0, n1), float("nan"), dtype=torch.float64, device="cuda")
    st = _lib().igamg_fd_apply_noalloc(n0, n1, C.c_void_p(U0.data_ptr()), C.c_void_p(U1.data_ptr()),
                                       C.c_void_p(Dinv.data_ptr()), C.c_void_p(R.data_ptr()), R.stride(0),
                                       tau, C.c_void_p(Z.data_ptr()), n1, None)
    assert st == 0, _lib().igamg_last_error(None)
    return Z


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def test_no_alloc_matches_scratch_entry_point_on_consecutive_calls():
    # two calls in a row on the shared array: a large tile, then a smaller one with
    # different data (stale contents of the first must not leak into the second)
    for seed, n0, n1, pad in ((1, 258, 259, 3), (2, 37, 21, 0), (3, 512, 512, 0)):
        U0, U1, Dinv, R = _tile(seed, n0, n1, pad)
        ref = _with_scratch(U0, U1, Dinv, R, n1, 0.25)
        got = _no_alloc(U0, U1, Dinv, R, n1, 0.25)
        torch.cuda.synchronize()
        assert torch.isfinite(got).all()
        assert _rel(got, ref) <= TOL


def test_no_alloc_rejects_tiles_beyond_its_limit():
    U0, U1, Dinv, R = _tile(4, 8, 8, 0)
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = _lib().igamg_fd_apply_noalloc(513, 512, C.c_void_p(U0.data_ptr()), C.c_void_p(U1.data_ptr()),
                                       C.c_void_p(Dinv.data_ptr()), C.c_void_p(R.data_ptr()), 512, 1.0,
                                       C.c_void_p(z.data_ptr()), 512, None)
    assert st == 1
    assert b"262144" in _lib().igamg_last_error(None)


def test_no_alloc_in_place_and_on_a_side_stream():
    """Z may be R itself (ldz == ldr, padded rows), and the call runs on the stream given:
    both against igamg_fd_apply on the same tile."""
    n0, n1, pad = 96, 70, 6
    U0, U1, Dinv, R = _tile(5, n0, n1, pad)
    ref = _with_scratch(U0, U1, Dinv, R, n1, 0.5)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        RZ = R.clone()
        st = _lib().igamg_fd_apply_noalloc(n0, n1, C.c_void_p(U0.data_ptr()), C.c_void_p(U1.data_ptr()),
                                           C.c_void_p(Dinv.data_ptr()), C.c_void_p(RZ.data_ptr()), RZ.stride(0),
                                           0.5, C.c_void_p(RZ.data_ptr()), RZ.stride(0), C.c_void_p(side.cuda_stream))
        assert st == 0, _lib().igamg_last_error(None)
    side.synchronize()
    assert _rel(RZ[:, :n1], ref) <= TOL
    assert torch.equal(RZ[:, n1:], R[:, n1:])      # the row padding is left alone
