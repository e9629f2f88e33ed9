"""ctypes binding of libigamg (include/igamg.h): same entry-point names, argument
marshalling only.  Device vectors are torch CUDA tensors (FP64, contiguous); the
library runs everything on the stream passed to igamg_setup.  There is no fallback: if
the shared library is missing the import of this module raises."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libigamg.so")

IGAMG_OK, IGAMG_ERR_NOT_CONVERGED = 0, 7
IGAMG_FP64, IGAMG_FP32, IGAMG_BF16 = 0, 1, 2
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_GEOMETRY", 3: "ERR_UNSUPPORTED", 4: "ERR_OOM",
          5: "ERR_CUDA", 6: "ERR_NUMERIC", 7: "ERR_NOT_CONVERGED", 8: "ERR_TIMEOUT"}


class igamg_problem(C.Structure):
    _fields_ = [("dim", C.c_int), ("num_patches", C.c_int),
                ("degree", C.POINTER(C.c_int)), ("num_knots", C.POINTER(C.c_int)),
                ("knots", C.POINTER(C.c_double)), ("geo_degree", C.POINTER(C.c_int)),
                ("geo_num_ctrl", C.POINTER(C.c_int)), ("geo_ctrl", C.POINTER(C.c_double)),
                ("side_bc", C.POINTER(C.c_int)), ("num_levels", C.c_int)]


class igamg_options(C.Structure):
    _fields_ = [("tau", C.c_double), ("sigma_scale", C.c_double), ("nu", C.c_int),
                ("mu", C.c_int), ("max_iter", C.c_int), ("precision", C.c_int), ("inner_tol", C.c_double),
                ("fd_engine", C.c_int),
                ("graphs", C.c_int),
                ("apply_engine", C.c_int),
                ("autotune", C.c_int),
                ("batch_engine", C.c_int)]


class igamg_result(C.Structure):
    _fields_ = [("iters", C.c_int), ("relres", C.c_double), ("t_setup_ms", C.c_double),
                ("t_assemble_ms", C.c_double), ("t_solve_ms", C.c_double), ("outer_iters", C.c_int)]


class igamg_request_info(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("relres", C.c_double), ("t_submit_ms", C.c_double),
                ("t_start_ms", C.c_double), ("t_done_ms", C.c_double), ("setup_ms", C.c_double), ("group", C.c_int)]


class igamg_server_counters(C.Structure):
    _fields_ = [("models", C.c_int), ("resident", C.c_int), ("device_bytes", C.c_int64), ("setups", C.c_int64),
                ("evictions", C.c_int64), ("completed", C.c_int64), ("waiting", C.c_int64), ("groups", C.c_int64),
                ("grouped", C.c_int64)]


def load_library(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libigamg.so not built ({path}); run __graft_entry__.build()")
    lib = C.CDLL(path)
    P = C.c_void_p
    sig = {
        "igamg_default_options": ([C.POINTER(igamg_options)], C.c_int),
        "igamg_setup": ([C.POINTER(igamg_problem), C.POINTER(igamg_options), P, C.POINTER(P)], C.c_int),
        "igamg_num_dofs": ([P, C.c_int, C.POINTER(C.c_int64)], C.c_int),
        "igamg_num_local": ([P, C.c_int, C.POINTER(C.c_int64)], C.c_int),
        "igamg_device_bytes": ([P, C.POINTER(C.c_int64)], C.c_int),
        "igamg_dof_map": ([P, C.c_int, C.POINTER(C.c_int64)], C.c_int),
        "igamg_rhs_from_coefs": ([P, P, P], C.c_int),
        "igamg_greville_points": ([P, C.c_int, P], C.c_int),
        "igamg_solve": ([P, P, P, C.c_double, C.POINTER(igamg_result)], C.c_int),
        "igamg_solve_host": ([P, P, P, C.c_double, C.POINTER(igamg_result)], C.c_int),
        "igamg_solve_multi": ([P, C.c_int, C.POINTER(P), C.POINTER(P), C.c_double, C.POINTER(igamg_result),
                               C.POINTER(C.c_int)], C.c_int),
        "igamg_apply": ([P, C.c_int, P, P], C.c_int),
        "igamg_smooth": ([P, C.c_int, P, P], C.c_int),
        "igamg_restrict": ([P, C.c_int, P, P], C.c_int),
        "igamg_prolong": ([P, C.c_int, P, P], C.c_int),
        "igamg_coarse_solve": ([P, P, P], C.c_int),
        "igamg_precondition": ([P, P, P], C.c_int),
        "igamg_cycle_time": ([P, P, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)], C.c_int),
        "igamg_sync": ([P], C.c_int),
        "igamg_profile_enable": ([P, C.c_int], C.c_int),
        "igamg_profile_read": ([P, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_double),
                                C.POINTER(C.c_double), C.POINTER(C.c_double)], C.c_int),
        "igamg_fd_apply": ([C.c_int, C.c_int, P, P, P, P, C.c_int, C.c_double, P, C.c_int, P, P], C.c_int),
        "igamg_fd_apply_noalloc": ([C.c_int, C.c_int, P, P, P, P, C.c_int, C.c_double, P, C.c_int, P],
                                   C.c_int),
        "igamg_micro_fp64": ([C.c_int, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_int)], C.c_int),
        "igamg_free": ([P], C.c_int),
        "igamg_last_error": ([P], C.c_char_p),
        "igamg_setup_batch": ([P, C.c_int, C.POINTER(igamg_options), C.c_int, P, C.POINTER(P)], C.c_int),
        "igamg_batch_context": ([P, C.c_int, C.POINTER(P)], C.c_int),
        "igamg_solve_batch": ([P, C.POINTER(P), C.POINTER(P), C.c_double, C.POINTER(igamg_result),
                               C.POINTER(C.c_int)], C.c_int),
        "igamg_free_batch": ([P], C.c_int),
        "igamg_batch_engine": ([P, C.POINTER(C.c_int), C.POINTER(C.c_int64), C.POINTER(C.c_double),
                                C.POINTER(C.c_double)], C.c_int),
        "igamg_server_create": ([C.POINTER(igamg_options), C.c_int, C.c_int64, C.POINTER(P)], C.c_int),
        "igamg_server_add_model": ([P, C.POINTER(igamg_problem), C.POINTER(C.c_int), C.POINTER(C.c_int64),
                                    C.POINTER(C.c_int64)], C.c_int),
        "igamg_server_submit": ([P, C.c_int, P, P, C.c_double, C.POINTER(C.c_int64)], C.c_int),
        "igamg_server_wait": ([P, C.c_int64, C.POINTER(igamg_request_info)], C.c_int),
        "igamg_server_stats": ([P, C.POINTER(igamg_server_counters)], C.c_int),
        "igamg_server_free": ([P], C.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


class IgamgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _ptr(t):
    if t is None:
        return None
    assert t.is_cuda and t.dtype.is_floating_point and t.is_contiguous(), "need a contiguous CUDA tensor"
    return C.c_void_p(t.data_ptr())


def _host_ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


class Problem:
    """igamg_problem built from any object with dim, degree (K,d), knots[k][j],
    corners (K, 2^d, d), side_bc (K, 2d) and num_levels; keeps the arrays alive."""

    def __init__(self, pr):
        K, d = np.asarray(pr.degree).shape
        self._deg = np.ascontiguousarray(np.asarray(pr.degree).ravel(), dtype=np.int32)
        kn = [np.asarray(pr.knots[k][j], dtype=np.float64) for k in range(K) for j in range(d)]
        self._nk = np.array([len(t) for t in kn], dtype=np.int32)
        self._kn = np.ascontiguousarray(np.concatenate(kn))
        self._gd = np.ones(K * d, dtype=np.int32)
        self._gn = np.full(K * d, 2, dtype=np.int32)
        self._ctrl = np.ascontiguousarray(np.asarray(pr.corners, dtype=np.float64).ravel())
        self._bc = np.ascontiguousarray(np.asarray(pr.side_bc).ravel(), dtype=np.int32)
        ip = lambda a: a.ctypes.data_as(C.POINTER(C.c_int))
        dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
        self.struct = igamg_problem(d, K, ip(self._deg), ip(self._nk), dp(self._kn), ip(self._gd),
                                    ip(self._gn), dp(self._ctrl), ip(self._bc), int(pr.num_levels))


def _stream_handle(stream):
    return C.c_void_p(stream.cuda_stream if stream is not None else 0)


def igamg_fd_apply(U0, U1, Dinv, R, tau, Z, scratch, stream=None):
    """Z = tau U0 ((U0^T R U1) .* Dinv) U1^T (2D row-major CUDA tensors, Z/R may be
    row-strided views); scratch holds >= 2 n0 n1 doubles."""
    n0, n1 = U0.shape[0], U1.shape[0]
    assert R.stride(1) == 1 and Z.stride(1) == 1
    st = lib().igamg_fd_apply(n0, n1, _ptr(U0), _ptr(U1), _ptr(Dinv), C.c_void_p(R.data_ptr()),
                              R.stride(0), tau, C.c_void_p(Z.data_ptr()), Z.stride(0), _ptr(scratch),
                              _stream_handle(stream))
    if st != IGAMG_OK:
        raise IgamgError(st, lib().igamg_last_error(None).decode())


def igamg_micro_fp64(kind=0, iters=1 << 16):
    """(TFLOP/s, SM count) of the FP64 FMA pipe (kind 0) or FP64 tensor-core MMAs (kind 1)."""
    tf, sms = C.c_double(), C.c_int()
    st = lib().igamg_micro_fp64(int(kind), int(iters), C.byref(tf), C.byref(sms))
    if st != IGAMG_OK:
        raise IgamgError(st, "igamg_micro_fp64 failed")
    return tf.value, sms.value


def igamg_default_options() -> igamg_options:
    o = igamg_options()
    lib().igamg_default_options(C.byref(o))
    return o


class Context:
    """Owns one igamg_ctx.  Methods are the ABI entry points without the igamg_ prefix."""

    @classmethod
    def borrowed(cls, handle, problem, stream):
        """Wrapper of a context owned elsewhere (a batch): free() leaves it alone."""
        self = cls.__new__(cls)
        self.problem = problem
        self.stream = stream
        self.h = handle
        self._borrowed = True
        return self

    def __init__(self, problem, options: igamg_options | None = None, stream=None):
        import torch
        self.problem = Problem(problem)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        st = lib().igamg_setup(C.byref(self.problem.struct), C.byref(options) if options else None,
                               C.c_void_p(stream.cuda_stream), C.byref(h))
        if st != IGAMG_OK:
            raise IgamgError(st, lib().igamg_last_error(None).decode())
        self.h = h

    def _check(self, st, allow_nc=False):
        if st == IGAMG_OK or (allow_nc and st == IGAMG_ERR_NOT_CONVERGED):
            return st
        raise IgamgError(st, lib().igamg_last_error(self.h).decode())

    def num_dofs(self, level=-1) -> int:
        n = C.c_int64()
        self._check(lib().igamg_num_dofs(self.h, level, C.byref(n)))
        return n.value

    def device_bytes(self) -> int:
        n = C.c_int64()
        self._check(lib().igamg_device_bytes(self.h, C.byref(n)))
        return n.value

    def num_local(self, level=-1) -> int:
        n = C.c_int64()
        self._check(lib().igamg_num_local(self.h, level, C.byref(n)))
        return n.value

    def dof_map(self, level=-1) -> np.ndarray:
        out = np.empty(self.num_local(level), dtype=np.int64)
        self._check(lib().igamg_dof_map(self.h, level, out.ctypes.data_as(C.POINTER(C.c_int64))))
        return out

    def greville_points(self, level=-1) -> np.ndarray:
        d = int(self.problem.struct.dim)
        out = np.empty((self.num_dofs(level), d))
        self._check(lib().igamg_greville_points(self.h, level, out.ctypes.data_as(C.c_void_p)))
        return out

    def rhs_from_coefs(self, coef, rhs):
        self._check(lib().igamg_rhs_from_coefs(self.h, _ptr(coef), _ptr(rhs)))

    def solve(self, rhs, x, tol=1e-8):
        res = igamg_result()
        st = self._check(lib().igamg_solve(self.h, _ptr(rhs), _ptr(x), tol, C.byref(res)), allow_nc=True)
        return res, st

    def solve_multi(self, rhs, xs, tol=1e-8):
        """Several right-hand sides of this problem together (igamg_solve_multi); rhs, xs:
        equal-length sequences of contiguous CUDA float64 tensors (xs: initial guesses in,
        solutions out).  Returns (overall status, [igamg_result], [status])."""
        n = len(rhs)
        assert len(xs) == n and n >= 1
        bp = (C.c_void_p * n)(*[_ptr(t) for t in rhs])
        xp = (C.c_void_p * n)(*[_ptr(t) for t in xs])
        res = (igamg_result * n)()
        sts = (C.c_int * n)()
        st = self._check(lib().igamg_solve_multi(self.h, n, bp, xp, tol, res, sts), allow_nc=True)
        return st, list(res), list(sts)

    def solve_host(self, rhs: np.ndarray, x: np.ndarray, tol=1e-8):
        res = igamg_result()
        st = self._check(lib().igamg_solve_host(self.h, _host_ptr(rhs), _host_ptr(x), tol, C.byref(res)),
                         allow_nc=True)
        return res, st

    def apply(self, level, x, y):
        self._check(lib().igamg_apply(self.h, level, _ptr(x), _ptr(y)))

    def smooth(self, level, r, z):
        self._check(lib().igamg_smooth(self.h, level, _ptr(r), _ptr(z)))

    def restrict(self, level, r, rc):
        self._check(lib().igamg_restrict(self.h, level, _ptr(r), _ptr(rc)))

    def prolong(self, level, uc, u):
        self._check(lib().igamg_prolong(self.h, level, _ptr(uc), _ptr(u)))

    def coarse_solve(self, r, x):
        self._check(lib().igamg_coarse_solve(self.h, _ptr(r), _ptr(x)))

    def precondition(self, r, z):
        self._check(lib().igamg_precondition(self.h, _ptr(r), _ptr(z)))

    def cycle_time(self, r, reps=10):
        """(ms per cycle, algorithmic bytes of one cycle) of the graph-replayed cycle in the
        context's working precision."""
        ms, by = C.c_double(), C.c_double()
        self._check(lib().igamg_cycle_time(self.h, _ptr(r), int(reps), C.byref(ms), C.byref(by)))
        return ms.value, by.value

    PROFILE_CLASSES = ("apply", "interior_fd", "interface", "transfer", "coarse", "vector")
    TENSOR_EXEC_CLASS = 6  # flops only: BF16 MMA work of the tensor-core FD
    TC_KERNEL_CLASS = 7    # sub-account of classes 1 and 2: the tensor-core kernel's launches

    def profile_enable(self, mask=0x3F):
        """mask: bit c times class c with CUDA events (0 disables profiling)."""
        self._check(lib().igamg_profile_enable(self.h, int(mask)))

    def profile_read(self):
        out = {}
        for i, name in list(enumerate(self.PROFILE_CLASSES)) + [(self.TENSOR_EXEC_CLASS, "tensor_exec"),
                                                                (self.TC_KERNEL_CLASS, "tc_kernel")]:
            n, ms, fl, by = C.c_int64(), C.c_double(), C.c_double(), C.c_double()
            self._check(lib().igamg_profile_read(self.h, i, C.byref(n), C.byref(ms), C.byref(fl), C.byref(by)))
            out[name] = {"launches": n.value, "ms": ms.value, "flops": fl.value, "bytes": by.value}
        return out

    def sync(self):
        self._check(lib().igamg_sync(self.h))

    def free(self):
        if getattr(self, "h", None):
            if not getattr(self, "_borrowed", False):
                lib().igamg_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Batch:
    """Owns one igamg_batch: independent problems set up together and solved concurrently
    by `workers` host threads with a CUDA stream each.  contexts[i] is problem i's context
    (borrowed: it lives as long as the batch)."""

    def __init__(self, problems, options: igamg_options | None = None, workers=0, stream=None):
        import torch
        self.problems = [Problem(p) for p in problems]
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        arr = (igamg_problem * len(self.problems))(*[p.struct for p in self.problems])
        self._arr = arr
        h = C.c_void_p()
        st = lib().igamg_setup_batch(arr, len(self.problems), C.byref(options) if options else None, int(workers),
                                     C.c_void_p(stream.cuda_stream), C.byref(h))
        if st != IGAMG_OK:
            raise IgamgError(st, lib().igamg_last_error(None).decode())
        self.h = h
        self.contexts = []
        for i, pr in enumerate(self.problems):
            ch = C.c_void_p()
            lib().igamg_batch_context(h, i, C.byref(ch))
            self.contexts.append(Context.borrowed(ch, pr, stream))

    def __len__(self):
        return len(self.contexts)

    def engine(self) -> str:
        """'lockstep' or 'streams': the engine igamg_solve_batch uses for this batch."""
        e = C.c_int()
        lib().igamg_batch_engine(self.h, C.byref(e), None, None, None)
        return "lockstep" if e.value == 0 else "streams"

    def stats(self):
        """Lockstep engine: kernel launches, algorithmic FLOPs and tensor-core MMA FLOPs of
        the last solve (None for worker streams)."""
        e, n, f, m = C.c_int(), C.c_int64(), C.c_double(), C.c_double()
        lib().igamg_batch_engine(self.h, C.byref(e), C.byref(n), C.byref(f), C.byref(m))
        if e.value != 0:
            return None
        return {"launches": n.value, "flops": f.value, "mma_flops": m.value}

    def solve(self, rhs, xs, tol=1e-8):
        """rhs, xs: sequences of contiguous CUDA float64 tensors (xs hold the initial guesses).
        Returns (overall status, [igamg_result], [status])."""
        n = len(self.contexts)
        assert len(rhs) == n and len(xs) == n
        bp = (C.c_void_p * n)(*[t.data_ptr() for t in rhs])
        xp = (C.c_void_p * n)(*[t.data_ptr() for t in xs])
        res = (igamg_result * n)()
        sts = (C.c_int * n)()
        st = lib().igamg_solve_batch(self.h, bp, xp, tol, res, sts)
        if st not in (IGAMG_OK, IGAMG_ERR_NOT_CONVERGED):
            bad = next(i for i in range(n) if sts[i] not in (IGAMG_OK, IGAMG_ERR_NOT_CONVERGED))
            raise IgamgError(st, f"problem {bad}: " + lib().igamg_last_error(self.contexts[bad].h).decode())
        return st, list(res), list(sts)

    def free(self):
        if getattr(self, "h", None):
            for c in self.contexts:
                c.h = None
            lib().igamg_free_batch(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Server:
    """Owns one igamg_server: models are registered problems, requests are load vectors
    (host float64 arrays in the model's dof order) answered by worker threads."""

    def __init__(self, options: igamg_options | None = None, workers=8, hbm_budget_bytes=64 << 30):
        h = C.c_void_p()
        st = lib().igamg_server_create(C.byref(options) if options else None, int(workers),
                                       int(hbm_budget_bytes), C.byref(h))
        if st != IGAMG_OK:
            raise IgamgError(st, lib().igamg_last_error(None).decode())
        self.h = h
        self._problems = []
        self._live = {}  # request id -> (rhs, x): kept alive until waited for

    def add_model(self, problem):
        """Returns (model id, number of dofs, estimated device bytes of its hierarchy)."""
        pr = Problem(problem)
        m, n, e = C.c_int(), C.c_int64(), C.c_int64()
        st = lib().igamg_server_add_model(self.h, C.byref(pr.struct), C.byref(m), C.byref(n), C.byref(e))
        if st != IGAMG_OK:
            raise IgamgError(st, lib().igamg_last_error(None).decode())
        self._problems.append(pr)
        return m.value, n.value, e.value

    def submit(self, model, rhs: np.ndarray, tol=1e-8):
        """Queues a solve; returns (request id, x) with x filled once waited for."""
        rhs = np.ascontiguousarray(rhs, dtype=np.float64)
        x = np.zeros_like(rhs)
        rid = C.c_int64()
        st = lib().igamg_server_submit(self.h, int(model), _host_ptr(rhs), _host_ptr(x), tol, C.byref(rid))
        if st != IGAMG_OK:
            raise IgamgError(st, "igamg_server_submit failed")
        self._live[rid.value] = (rhs, x)
        return rid.value, x

    def wait(self, request):
        info = igamg_request_info()
        st = lib().igamg_server_wait(self.h, int(request), C.byref(info))
        if st != IGAMG_OK:
            raise IgamgError(st, "igamg_server_wait: unknown request")
        self._live.pop(request, None)
        return {f: getattr(info, f) for f, _ in info._fields_}

    def stats(self):
        s = igamg_server_counters()
        lib().igamg_server_stats(self.h, C.byref(s))
        return {f: getattr(s, f) for f, _ in s._fields_}

    def free(self):
        if getattr(self, "h", None):
            lib().igamg_server_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
