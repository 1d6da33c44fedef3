"""ctypes binding of libpdmcf.so (the C ABI declared in include/pdmcf.h).

Argument marshalling only: every step of a solve runs in the library's CUDA kernels.
The functions carry the C names; ``Problem`` is a small owner of a problem handle.
Importing this module fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

MCF_OK = 0
MCF_PENDING = 1
MCF_ERR_INVALID = -1
MCF_ERR_NOT_CONNECTED = -2
MCF_ERR_OOM = -3
MCF_ERR_CUDA = -4
MCF_ERR_NUMERIC = -5
MCF_ERR_NOT_CONVERGED = -6
MCF_ERR_TIMEOUT = -7
MCF_ERR_BUSY = -8
MCF_ERR_OOM_BUDGET = -9
MCF_ERR_CANCELLED = -10

MCF_LOG, MCF_POW = 0, 1
MCF_FP32, MCF_FP64, MCF_BF16_F = 0, 1, 2
MCF_STOP_PAPER, MCF_STOP_REL_KKT, MCF_STOP_NONE = 0, 1, 2

PRECISIONS = {"fp32": MCF_FP32, "fp64": MCF_FP64, "bf16": MCF_BF16_F}
STOP_MODES = {"paper": MCF_STOP_PAPER, "kkt": MCF_STOP_REL_KKT, "none": MCF_STOP_NONE}


class mcf_options(C.Structure):
    _fields_ = [
        ("eps", C.c_double), ("stop_mode", C.c_int), ("max_iters", C.c_int64),
        ("rho", C.c_double), ("theta", C.c_double), ("k_adapt", C.c_int),
        ("tau", C.c_double), ("omega_freeze_iter", C.c_int64), ("k_check", C.c_int),
        ("precision", C.c_int), ("warm_start", C.c_int), ("polish_iters", C.c_int),
        ("use_graphs", C.c_int), ("device", C.c_int), ("cuda_stream", C.c_void_p),
        ("omega0", C.c_double), ("stall_checks", C.c_int), ("compensated_duals", C.c_int),
        ("autotune", C.c_int), ("shape", C.c_int), ("adapt_guard", C.c_double),
        ("adapt_guard_below", C.c_double), ("check_log", C.c_char_p),
    ]


class mcf_result(C.Structure):
    _fields_ = [
        ("T", C.POINTER(C.c_double)), ("F", C.POINTER(C.c_double)), ("Y", C.POINTER(C.c_double)),
        ("iters", C.c_int64), ("status", C.c_int), ("feasible", C.c_int),
        ("utility", C.c_double), ("dual_bound", C.c_double), ("r", C.c_double),
        ("r_over_nm", C.c_double), ("rel_gap", C.c_double), ("rel_cons", C.c_double),
        ("rel_stat", C.c_double), ("rel_kkt", C.c_double), ("nonpos_frac", C.c_double),
        ("omega", C.c_double), ("stalled", C.c_int), ("delta_f", C.c_double),
        ("delta_y", C.c_double), ("omega_frozen_at", C.c_int64), ("seconds", C.c_double),
    ]


class mcf_kernel_times(C.Structure):
    _fields_ = [("ms", C.c_double * 4), ("launches", C.c_int64 * 4), ("ms_total", C.c_double),
                ("shape", C.c_int)]


KERNEL_KINDS = ("edge", "node", "check", "scalar")

SYMBOLS = [
    "mcf_create_problem", "mcf_update_capacities", "mcf_update_weights",
    "mcf_destroy_problem", "mcf_problem_size", "mcf_problem_node_order", "mcf_problem_edge_order",
    "mcf_problem_device_bytes",
    "mcf_options_default", "mcf_solve", "mcf_solve_timed", "mcf_solve_batch", "mcf_autotune",
    "mcf_submit", "mcf_poll", "mcf_wait",
    "mcf_cancel", "mcf_serving_config", "mcf_serving_shutdown", "mcf_project_capped_simplex",
    "mcf_project_capped_simplex_noalloc", "mcf_shape_info", "mcf_test_withhold_next_copy",
    "mcf_save_state", "mcf_load_state",
    "mcf_last_error", "mcf_version",
]


def _load() -> C.CDLL:
    path = _build.LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"libpdmcf.so is not built ({path}); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'` first")
    lib = C.CDLL(path)
    P = C.c_void_p
    dp = C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int32)
    sig = {
        "mcf_create_problem": (C.c_int, [C.c_int32, C.c_int32, ip, ip, dp, C.c_int, dp, dp,
                                         C.c_int64, C.POINTER(P)]),
        "mcf_update_capacities": (C.c_int, [P, dp]),
        "mcf_update_weights": (C.c_int, [P, dp]),
        "mcf_destroy_problem": (C.c_int, [P]),
        "mcf_problem_size": (C.c_int, [P, ip, ip]),
        "mcf_problem_node_order": (C.c_int, [P, ip]),
        "mcf_problem_edge_order": (C.c_int, [P, ip]),
        "mcf_problem_device_bytes": (C.c_int64, [P, C.c_int]),
        "mcf_options_default": (None, [C.POINTER(mcf_options)]),
        "mcf_solve": (C.c_int, [P, C.POINTER(mcf_options), C.POINTER(mcf_result)]),
        "mcf_solve_timed": (C.c_int, [P, C.POINTER(mcf_options), C.POINTER(mcf_result),
                                      C.POINTER(mcf_kernel_times)]),
        "mcf_solve_batch": (C.c_int, [C.POINTER(P), C.c_int, C.POINTER(mcf_options),
                                      C.POINTER(mcf_result)]),
        "mcf_autotune": (C.c_int, [P, C.POINTER(mcf_options), C.POINTER(C.c_int),
                                   C.POINTER(C.c_double)]),
        "mcf_submit": (C.c_int, [P, C.POINTER(mcf_options), C.POINTER(C.c_int64)]),
        "mcf_poll": (C.c_int, [C.c_int64, C.POINTER(C.c_int), C.POINTER(mcf_result)]),
        "mcf_wait": (C.c_int, [C.c_int64, C.c_int64, C.POINTER(C.c_int), C.POINTER(mcf_result)]),
        "mcf_cancel": (C.c_int, [C.c_int64]),
        "mcf_serving_config": (C.c_int, [C.c_int64, C.c_int]),
        "mcf_serving_shutdown": (C.c_int, []),
        "mcf_test_withhold_next_copy": (C.c_int, []),
        "mcf_save_state": (C.c_int, [P, C.c_char_p]),
        "mcf_load_state": (C.c_int, [P, C.c_char_p, C.c_int]),
        "mcf_project_capped_simplex": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, P, P, P, P,
                                                 dp, P]),
        "mcf_project_capped_simplex_noalloc": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, P, P, P,
                                                         P, dp, P]),
        "mcf_shape_info": (C.c_int, [ip, ip, ip, ip]),
        "mcf_last_error": (C.c_char_p, []),
        "mcf_version": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


LIB = _load()


class MCFError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where} failed with {code}: {mcf_last_error()}")


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


# ---------------------------------------------------------------- C-named functions

def mcf_last_error() -> str:
    return LIB.mcf_last_error().decode()


def mcf_version() -> str:
    return LIB.mcf_version().decode()


def mcf_shape_info() -> list[tuple[int, int, int, int]]:
    """[(group, vpt, block, kind)] per shape index (kind 0 register, 1 bulk-copy pipelined,
    2 register with in-sums)."""
    cnt = LIB.mcf_shape_info(None, None, None, None)
    g = (C.c_int32 * cnt)()
    v = (C.c_int32 * cnt)()
    b = (C.c_int32 * cnt)()
    t = (C.c_int32 * cnt)()
    LIB.mcf_shape_info(g, v, b, t)
    return [(g[i], v[i], b[i], t[i]) for i in range(cnt)]


def mcf_options_default(**overrides) -> mcf_options:
    o = mcf_options()
    LIB.mcf_options_default(C.byref(o))
    for k, v in overrides.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        if k == "stop_mode" and isinstance(v, str):
            v = STOP_MODES[v]
        if k == "check_log" and isinstance(v, str):
            v = v.encode()
        setattr(o, k, v)
    return o


def mcf_create_problem(n, tail, head, cap, kind, w, gamma=None) -> C.c_void_p:
    tail = np.ascontiguousarray(tail, dtype=np.int32)
    head = np.ascontiguousarray(head, dtype=np.int32)
    cap = np.ascontiguousarray(cap, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    k = MCF_LOG if kind in ("log", MCF_LOG) else MCF_POW
    if gamma is None:
        g, glen = None, 0
    else:
        g = np.ascontiguousarray(np.atleast_1d(np.asarray(gamma, dtype=np.float64)).ravel())
        glen = g.size
    h = C.c_void_p()
    rc = LIB.mcf_create_problem(int(n), int(tail.size), _iptr(tail), _iptr(head), _dptr(cap), k,
                                _dptr(w), _dptr(g) if g is not None else None, glen, C.byref(h))
    if rc != MCF_OK:
        raise MCFError(rc, "mcf_create_problem")
    return h


def mcf_destroy_problem(h) -> None:
    rc = LIB.mcf_destroy_problem(h)
    if rc != MCF_OK:
        raise MCFError(rc, "mcf_destroy_problem")


def mcf_update_capacities(h, cap) -> None:
    cap = np.ascontiguousarray(cap, dtype=np.float64)
    rc = LIB.mcf_update_capacities(h, _dptr(cap))
    if rc != MCF_OK:
        raise MCFError(rc, "mcf_update_capacities")


def mcf_update_weights(h, w) -> None:
    w = np.ascontiguousarray(w, dtype=np.float64)
    rc = LIB.mcf_update_weights(h, _dptr(w))
    if rc != MCF_OK:
        raise MCFError(rc, "mcf_update_weights")


def mcf_problem_device_bytes(h, precision=MCF_FP32) -> int:
    return int(LIB.mcf_problem_device_bytes(h, PRECISIONS.get(precision, precision)))


def _result_struct(n, m, want_T, want_F, want_Y):
    res = mcf_result()
    bufs = {}
    if want_T:
        bufs["T"] = np.zeros((n, n))
        res.T = _dptr(bufs["T"])
    if want_F:
        bufs["F"] = np.zeros((n, m))
        res.F = _dptr(bufs["F"])
    if want_Y:
        bufs["Y"] = np.zeros((n, n))
        res.Y = _dptr(bufs["Y"])
    return res, bufs


def _result_dict(res: mcf_result, bufs: dict) -> dict:
    out = {f: getattr(res, f) for f, _ in mcf_result._fields_ if f not in ("T", "F", "Y")}
    out.update(bufs)
    return out


def mcf_solve(h, opts: mcf_options, n, m, want_T=True, want_F=False, want_Y=False,
              raise_on_error=True) -> dict:
    res, bufs = _result_struct(n, m, want_T, want_F, want_Y)
    rc = LIB.mcf_solve(h, C.byref(opts), C.byref(res))
    if raise_on_error and rc not in (MCF_OK, MCF_ERR_NOT_CONVERGED):
        raise MCFError(rc, "mcf_solve")
    out = _result_dict(res, bufs)
    out["rc"] = rc
    return out


def mcf_solve_timed(h, opts: mcf_options, n, m, want_T=False) -> tuple[dict, dict]:
    """Returns (result dict, per-kernel times {kind: (ms_total, launches)} + 'ms_total')."""
    res, bufs = _result_struct(n, m, want_T, False, False)
    kt = mcf_kernel_times()
    rc = LIB.mcf_solve_timed(h, C.byref(opts), C.byref(res), C.byref(kt))
    if rc not in (MCF_OK, MCF_ERR_NOT_CONVERGED):
        raise MCFError(rc, "mcf_solve_timed")
    times = {k: (kt.ms[i], int(kt.launches[i])) for i, k in enumerate(KERNEL_KINDS)}
    times["ms_total"] = kt.ms_total
    out = _result_dict(res, bufs)
    out["rc"] = rc
    out["shape"] = kt.shape
    return out, times


def mcf_solve_batch(problems, opts: mcf_options, want_T=False, want_Y=False) -> tuple[int, list]:
    """problems: list of Problem. Returns (rc, [result dict per problem])."""
    k = len(problems)
    hs = (C.c_void_p * k)(*[p.h for p in problems])
    results = (mcf_result * k)()
    bufs = []
    for i, p in enumerate(problems):
        r, b = _result_struct(p.n, p.m, want_T, False, want_Y)
        results[i] = r
        bufs.append(b)
    rc = LIB.mcf_solve_batch(hs, k, C.byref(opts), results)
    if rc not in (MCF_OK, MCF_ERR_NOT_CONVERGED):
        raise MCFError(rc, "mcf_solve_batch")
    return rc, [_result_dict(results[i], bufs[i]) for i in range(k)]


def mcf_autotune(h, opts: mcf_options) -> tuple[int, float]:
    """Returns (fastest shape index, ms per iteration)."""
    shape = C.c_int(-1)
    ms = C.c_double(0.0)
    rc = LIB.mcf_autotune(h, C.byref(opts), C.byref(shape), C.byref(ms))
    if rc != MCF_OK:
        raise MCFError(rc, "mcf_autotune")
    return shape.value, ms.value


def mcf_submit(h, opts: mcf_options) -> int:
    t = C.c_int64()
    rc = LIB.mcf_submit(h, C.byref(opts), C.byref(t))
    if rc != MCF_OK:
        raise MCFError(rc, "mcf_submit")
    return t.value


def mcf_poll(ticket: int, n=0, m=0, want_T=False, want_F=False, want_Y=False):
    """Returns None while pending, else the result dict (with 'status')."""
    res, bufs = _result_struct(n, m, want_T, want_F, want_Y)
    st = C.c_int()
    rc = LIB.mcf_poll(ticket, C.byref(st), C.byref(res))
    if rc == MCF_PENDING:
        return None
    if rc != MCF_OK:
        raise MCFError(rc, "mcf_poll")
    out = _result_dict(res, bufs)
    out["status"] = st.value
    return out


def mcf_wait(ticket: int, timeout_ms=-1, n=0, m=0, want_T=False, want_F=False, want_Y=False):
    res, bufs = _result_struct(n, m, want_T, want_F, want_Y)
    st = C.c_int()
    rc = LIB.mcf_wait(ticket, int(timeout_ms), C.byref(st), C.byref(res))
    if rc == MCF_ERR_TIMEOUT:
        return None
    if rc != MCF_OK:
        raise MCFError(rc, "mcf_wait")
    out = _result_dict(res, bufs)
    out["status"] = st.value
    return out


def mcf_cancel(ticket: int) -> None:
    rc = LIB.mcf_cancel(ticket)
    if rc != MCF_OK:
        raise MCFError(rc, "mcf_cancel")


def mcf_project_capped_simplex(n: int, m: int, ld: int, Qt_ptr: int, cap_ptr: int, Ft_ptr: int,
                               mu_ptr: int, stream: int = 0) -> float:
    """Device pointers (ints, e.g. torch tensor.data_ptr()); returns sum ||F - Q||^2."""
    d2 = C.c_double(0.0)
    rc = LIB.mcf_project_capped_simplex(int(n), int(m), int(ld), Qt_ptr, cap_ptr, Ft_ptr, mu_ptr,
                                        C.byref(d2), stream or None)
    if rc != MCF_OK:
        raise MCFError(rc, "mcf_project_capped_simplex")
    return d2.value


def mcf_project_capped_simplex_noalloc(n: int, m: int, ld: int, Qt_ptr: int, cap_ptr: int,
                                       Ft_ptr: int, mu_ptr: int, stream: int = 0,
                                       want_dist2: bool = True):
    """As mcf_project_capped_simplex, for callers that cannot allocate device memory (the
    scratch is a fixed array in the library; m <= 262144). Returns sum ||F - Q||^2, or None
    with want_dist2=False: then dist2 is passed as NULL and the call returns as soon as the
    work is queued on `stream`."""
    d2 = C.c_double(0.0)
    rc = LIB.mcf_project_capped_simplex_noalloc(int(n), int(m), int(ld), Qt_ptr, cap_ptr, Ft_ptr,
                                                mu_ptr, C.byref(d2) if want_dist2 else None,
                                                stream or None)
    if rc != MCF_OK:
        raise MCFError(rc, "mcf_project_capped_simplex_noalloc")
    return d2.value if want_dist2 else None


def mcf_serving_config(hbm_budget_bytes: int, max_resident: int) -> None:
    rc = LIB.mcf_serving_config(int(hbm_budget_bytes), int(max_resident))
    if rc != MCF_OK:
        raise MCFError(rc, "mcf_serving_config")


def mcf_test_withhold_next_copy() -> None:
    """Testing aid: the next bulk-copy pipelined solve has one stage whose copies never come,
    so its bounded device wait runs out (see the header)."""
    rc = LIB.mcf_test_withhold_next_copy()
    if rc != MCF_OK:
        raise MCFError(rc, "mcf_test_withhold_next_copy")


def mcf_serving_shutdown() -> None:
    rc = LIB.mcf_serving_shutdown()
    if rc != MCF_OK:
        raise MCFError(rc, "mcf_serving_shutdown")


# ---------------------------------------------------------------- convenience owner

class Problem:
    """Owns an mcf_problem handle built from an instance-like object (n, tail, head, cap,
    kind, w, gamma)."""

    def __init__(self, inst):
        self.n = int(inst.n)
        self.m = int(len(inst.tail))
        self.h = mcf_create_problem(inst.n, inst.tail, inst.head, inst.cap, inst.kind, inst.w,
                                    inst.gamma)

    def solve(self, want_T=True, want_F=False, want_Y=False, raise_on_error=True, **opts) -> dict:
        return mcf_solve(self.h, mcf_options_default(**opts), self.n, self.m, want_T, want_F,
                         want_Y, raise_on_error)

    def solve_timed(self, want_T=False, **opts):
        return mcf_solve_timed(self.h, mcf_options_default(**opts), self.n, self.m, want_T)

    def autotune(self, **opts) -> tuple[int, float]:
        return mcf_autotune(self.h, mcf_options_default(**opts))

    def submit(self, **opts) -> int:
        return mcf_submit(self.h, mcf_options_default(**opts))

    def save_state(self, path: str) -> None:
        rc = LIB.mcf_save_state(self.h, os.fsencode(path))
        if rc != MCF_OK:
            raise MCFError(rc, "mcf_save_state")

    def load_state(self, path: str, device: int = 0) -> None:
        rc = LIB.mcf_load_state(self.h, os.fsencode(path), int(device))
        if rc != MCF_OK:
            raise MCFError(rc, "mcf_load_state")

    def update_capacities(self, cap):
        mcf_update_capacities(self.h, cap)

    def update_weights(self, w):
        mcf_update_weights(self.h, w)

    def device_bytes(self, precision="fp32") -> int:
        return mcf_problem_device_bytes(self.h, precision)

    def node_order(self) -> tuple[bool, np.ndarray]:
        """(renumbered, node_of): node_of[caller node] = the library's internal node."""
        out = np.empty(self.n, dtype=np.int32)
        rc = LIB.mcf_problem_node_order(self.h, out.ctypes.data_as(C.POINTER(C.c_int32)))
        if rc < 0:
            raise MCFError(rc, "mcf_problem_node_order")
        return bool(rc), out

    def edge_order(self) -> np.ndarray:
        """edge_of[internal edge] = the caller's edge index (rows of F in a saved state)."""
        out = np.empty(self.m, dtype=np.int32)
        rc = LIB.mcf_problem_edge_order(self.h, out.ctypes.data_as(C.POINTER(C.c_int32)))
        if rc != MCF_OK:
            raise MCFError(rc, "mcf_problem_edge_order")
        return out

    def close(self):
        if self.h:
            mcf_destroy_problem(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
