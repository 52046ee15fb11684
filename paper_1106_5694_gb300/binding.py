"""Thin Python binding of the C ABI in include/dgs.h (argument marshalling only).

Every function has the name of the C entry point it calls.  Device arrays are
torch CUDA tensors (int32, contiguous); the stream defaults to torch's current
stream on the tensors' device.  There is no fallback: if the CUDA library is
not built, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libdgs.so")

DGS_OK = 0
DGS_ERR_INVALID = 1
DGS_ERR_RANGE = 2
DGS_ERR_OOM = 3
DGS_ERR_CUDA = 4
DGS_TIMEOUT = 5
DGS_PENDING = 6
DGS_ERR_BUSY = 7
DGS_ERR_INTERNAL = 8
DGS_CANCELLED = 9

DGS_INIT_GREEDY = 0
DGS_INIT_RANDOM = 1
DGS_INIT_IDENTITY = 2
DGS_INIT_USER = 3
DGS_REEVAL_BOX = 0
DGS_REEVAL_ALL = 1
DGS_ALG_PARALLEL = 0
DGS_ALG_SEQUENTIAL = 1
DGS_EVAL_TILE_PAIRS = 0
DGS_EVAL_ROW_OWNER = 1

EXPORTED = ["dgs_default_options", "dgs_solve", "dgs_solve_ex", "dgs_solve_host", "dgs_evaluate",
            "dgs_evaluate_static", "dgs_greedy_init", "dgs_status_string", "dgs_last_cuda_error",
            "dgs_solve_batched", "dgs_server_create", "dgs_server_request_bytes", "dgs_submit", "dgs_poll",
            "dgs_server_wait", "dgs_server_get_info", "dgs_server_destroy", "dgs_autotune", "dgs_get_tuning",
            "dgs_submit_ex", "dgs_solve_rect", "dgs_read_bandwidth",
            "dgs_release_cached_memory", "dgs_cancel"]
DGS_STATIC_MAX_N = 8192
DGS_BATCH_MAX_N = 32767
DGS_SUBMIT_HOST = 1


class dgs_options(ctypes.Structure):
    _fields_ = [
        ("init", ctypes.c_int32),
        ("init_sigma", ctypes.c_void_p),
        ("max_sweeps", ctypes.c_int32),
        ("deadline_us", ctypes.c_int64),
        ("trace_capacity", ctypes.c_int32),
        ("trace_accepted", ctypes.c_void_p),
        ("trace_applied", ctypes.c_void_p),
        ("trace_objective", ctypes.c_void_p),
        ("profile", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("reeval_rule", ctypes.c_int32),
        ("algorithm", ctypes.c_int32),
        ("evaluation", ctypes.c_int32),
        ("status_out", ctypes.c_void_p),
    ]


class dgs_stats(ctypes.Structure):
    _fields_ = [
        ("sweeps", ctypes.c_int32),
        ("events", ctypes.c_int32),
        ("swaps_applied", ctypes.c_int64),
        ("greedy_rounds", ctypes.c_int32),
        ("full_evaluations", ctypes.c_int32),
        ("row_updates", ctypes.c_int32),
        ("rows_recomputed", ctypes.c_int64),
        ("initial_objective", ctypes.c_int64),
        ("kernel_launches", ctypes.c_int64),
        ("evaluation_ms", ctypes.c_double),
        ("greedy_ms", ctypes.c_double),
        ("greedy_rescans", ctypes.c_int64),
        ("status", ctypes.c_int32),
        ("solve_ms", ctypes.c_double),
    ]

    def as_dict(self):
        return {name: (float if name.endswith("_ms") else int)(getattr(self, name)) for name, _ in self._fields_}


class dgs_request_times(ctypes.Structure):
    _fields_ = [("submit_ns", ctypes.c_int64), ("admit_ns", ctypes.c_int64), ("done_ns", ctypes.c_int64),
                ("upload_ns", ctypes.c_int64), ("ready_ns", ctypes.c_int64), ("start_ns", ctypes.c_int64)]


class dgs_server_info(ctypes.Structure):
    _fields_ = [
        ("resident", ctypes.c_int32),
        ("queued", ctypes.c_int32),
        ("steps", ctypes.c_int64),
        ("completed", ctypes.c_int64),
        ("bytes_in_use", ctypes.c_size_t),
        ("kernel_launches", ctypes.c_int64),
        ("upload_ms", ctypes.c_double),
        ("step_ms", ctypes.c_double),
    ]


class dgs_tuning(ctypes.Structure):
    _fields_ = [
        ("n_lo", ctypes.c_int32),
        ("n_hi", ctypes.c_int32),
        ("rows_per_thread", ctypes.c_int32),
        ("strip", ctypes.c_int32),
        ("best_ms", ctypes.c_double),
        ("candidates", ctypes.c_int32),
        ("cand_rows", ctypes.c_int32 * 16),
        ("cand_strip", ctypes.c_int32 * 16),
        ("cand_ms", ctypes.c_double * 16),
        ("tma", ctypes.c_int32),
        ("cand_tma", ctypes.c_int32 * 16),
    ]


_lib = None


def library_path() -> str:
    return _LIB_PATH


def load():
    """Load libdgs.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {_LIB_PATH} is missing "
                           "(run __graft_entry__.build() or paper_1106_5694_gb300/build_ext.py)")
    lib = ctypes.CDLL(_LIB_PATH)
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.dgs_default_options.argtypes = [ctypes.POINTER(dgs_options)]
    lib.dgs_default_options.restype = None
    lib.dgs_solve.argtypes = [P, i32, P, ctypes.POINTER(i64), P]
    lib.dgs_solve.restype = ctypes.c_int
    # objective_out may be host (byref int64) or device memory (a pointer)
    lib.dgs_solve_ex.argtypes = [P, i32, P, P, ctypes.POINTER(dgs_options), ctypes.POINTER(dgs_stats), P]
    lib.dgs_solve_ex.restype = ctypes.c_int
    lib.dgs_solve_host.argtypes = [P, i32, P, ctypes.POINTER(i64), ctypes.POINTER(dgs_options),
                                   ctypes.POINTER(dgs_stats), P]
    lib.dgs_solve_host.restype = ctypes.c_int
    lib.dgs_evaluate.argtypes = [P, i32, P, P, P, P, P, P]
    lib.dgs_evaluate.restype = ctypes.c_int
    lib.dgs_evaluate_static.argtypes = [P, i32, P, P, P, P, P, P]
    lib.dgs_evaluate_static.restype = ctypes.c_int
    lib.dgs_greedy_init.argtypes = [P, i32, P, P]
    lib.dgs_greedy_init.restype = ctypes.c_int
    lib.dgs_status_string.argtypes = [ctypes.c_int]
    lib.dgs_status_string.restype = ctypes.c_char_p
    lib.dgs_last_cuda_error.argtypes = []
    lib.dgs_last_cuda_error.restype = ctypes.c_char_p
    lib.dgs_solve_batched.argtypes = [P, P, i32, P, P, ctypes.POINTER(dgs_options), P, P, P]
    lib.dgs_solve_batched.restype = ctypes.c_int
    lib.dgs_server_create.argtypes = [ctypes.c_size_t, i32, ctypes.POINTER(ctypes.c_void_p)]
    lib.dgs_server_create.restype = ctypes.c_int
    lib.dgs_server_request_bytes.argtypes = [i32]
    lib.dgs_server_request_bytes.restype = ctypes.c_size_t
    lib.dgs_submit.argtypes = [P, P, i32, i32, ctypes.POINTER(ctypes.c_uint64)]
    lib.dgs_submit.restype = ctypes.c_int
    lib.dgs_submit_ex.argtypes = [P, P, i32, i32, ctypes.POINTER(dgs_options), ctypes.POINTER(ctypes.c_uint64)]
    lib.dgs_submit_ex.restype = ctypes.c_int
    lib.dgs_poll.argtypes = [P, ctypes.c_uint64, P, ctypes.POINTER(i64), ctypes.POINTER(dgs_stats),
                             ctypes.POINTER(dgs_request_times)]
    lib.dgs_poll.restype = ctypes.c_int
    lib.dgs_server_wait.argtypes = [P, ctypes.c_uint64, i64, P, ctypes.POINTER(i64), ctypes.POINTER(dgs_stats),
                                    ctypes.POINTER(dgs_request_times)]
    lib.dgs_server_wait.restype = ctypes.c_int
    lib.dgs_cancel.argtypes = [P, ctypes.c_uint64]
    lib.dgs_cancel.restype = ctypes.c_int
    lib.dgs_server_get_info.argtypes = [P, ctypes.POINTER(dgs_server_info)]
    lib.dgs_server_get_info.restype = ctypes.c_int
    lib.dgs_server_destroy.argtypes = [P]
    lib.dgs_server_destroy.restype = None
    lib.dgs_solve_rect.argtypes = [P, i32, i32, P, ctypes.POINTER(i64), ctypes.POINTER(dgs_options),
                                   ctypes.POINTER(dgs_stats), P]
    lib.dgs_solve_rect.restype = ctypes.c_int
    lib.dgs_autotune.argtypes = [i32, ctypes.POINTER(dgs_tuning), P]
    lib.dgs_autotune.restype = ctypes.c_int
    lib.dgs_get_tuning.argtypes = [i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.dgs_get_tuning.restype = ctypes.c_int
    lib.dgs_read_bandwidth.argtypes = [P, ctypes.c_size_t, i32, ctypes.POINTER(ctypes.c_double), P]
    lib.dgs_read_bandwidth.restype = ctypes.c_int
    lib.dgs_release_cached_memory.argtypes = []
    lib.dgs_release_cached_memory.restype = ctypes.c_int
    _lib = lib
    return lib


def _dev(t: torch.Tensor, name: str) -> ctypes.c_void_p:
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.int32 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous int32 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(t: torch.Tensor, stream):
    s = stream if stream is not None else torch.cuda.current_stream(t.device)
    return ctypes.c_void_p(s.cuda_stream)


def _n(benefit) -> int:
    if benefit.ndim != 2 or benefit.shape[0] != benefit.shape[1]:
        raise ValueError("benefit must be a square n x n matrix")
    return int(benefit.shape[0])


def dgs_status_string(status: int) -> str:
    return load().dgs_status_string(int(status)).decode()


def dgs_last_cuda_error() -> str:
    return load().dgs_last_cuda_error().decode()


def dgs_default_options() -> dgs_options:
    o = dgs_options()
    load().dgs_default_options(ctypes.byref(o))
    return o


def _options(init=DGS_INIT_GREEDY, init_sigma=None, max_sweeps=0, deadline_us=0, trace=None, profile=0, seed=0,
             reeval=DGS_REEVAL_BOX, algorithm=DGS_ALG_PARALLEL, evaluation=DGS_EVAL_TILE_PAIRS):
    o = dgs_default_options()
    o.algorithm = int(algorithm)
    o.evaluation = int(evaluation)
    o.init = init
    o.seed = int(seed)
    o.reeval_rule = int(reeval)
    o.profile = int(profile)
    o.init_sigma = _dev(init_sigma, "init_sigma") if init_sigma is not None else None
    o.max_sweeps = max_sweeps
    o.deadline_us = deadline_us
    if trace is not None:
        acc, app, obj = trace
        o.trace_capacity = int(acc.numel())
        o.trace_accepted = ctypes.c_void_p(acc.data_ptr())
        o.trace_applied = ctypes.c_void_p(app.data_ptr())
        o.trace_objective = ctypes.c_void_p(obj.data_ptr())
    return o


def _wait(benefit, stream):
    (stream if stream is not None else torch.cuda.current_stream(benefit.device)).synchronize()


# Host memory that the library's stream callbacks of solves enqueued with
# wait=False still have to write (objective, stats), each entry kept with an
# event recorded after its solve until that event has completed: a caller may
# drop the Pending at once.
_IN_FLIGHT = []


def _keep_until_done(benefit, stream, objs):
    _IN_FLIGHT[:] = [x for x in _IN_FLIGHT if not x[0].query()]
    ev = torch.cuda.Event()
    ev.record(stream if stream is not None else torch.cuda.current_stream(benefit.device))
    _IN_FLIGHT.append((ev, objs))


class Pending:
    """A stream-ordered solve in flight (wait=False): result() waits for the
    stream and returns what the waiting form returns."""

    def __init__(self, st, benefit, stream, out, f, stats=None, options=None, stats_dict=True, wait=True):
        self._st, self._benefit, self._stream = st, benefit, stream
        self._out, self._f, self._stats, self._options = out, f, stats, options
        self._stats_dict = stats_dict
        if st == DGS_OK and not wait:
            _keep_until_done(benefit, stream, (f, stats, options))

    def result(self):
        if self._st == DGS_OK:
            _wait(self._benefit, self._stream)
        if self._stats is None:
            if self._stats_dict:
                return self._st, self._out, int(self._f.value), {}
            return self._st, self._out, int(self._f.value)
        st = int(self._stats.status) if self._st == DGS_OK else self._st
        return st, self._out, int(self._f.value), self._stats.as_dict()


def dgs_solve(benefit: torch.Tensor, sigma_out: torch.Tensor | None = None, stream=None, wait=True):
    """dgs_solve (stream-ordered): returns (status of the call, sigma_out,
    objective).  With wait (default) the stream is synchronised first, so the
    objective is final; with wait=False a Pending whose result() does that.
    The solve's own outcome (range error, ...) is not reported by this entry
    point: after a device-side error every sigma_out entry is -1, and
    dgs_solve_ex reports the outcome."""
    n = _n(benefit)
    if sigma_out is None:
        sigma_out = torch.empty(n, dtype=torch.int32, device=benefit.device)
    f = ctypes.c_int64(0)
    st = load().dgs_solve(_dev(benefit, "benefit"), n, _dev(sigma_out, "sigma_out"), ctypes.byref(f),
                          _stream(benefit, stream))
    pending = Pending(st, benefit, stream, sigma_out, f, stats_dict=False, wait=wait)
    return pending.result() if wait else pending


def dgs_solve_ex(benefit: torch.Tensor, sigma_out: torch.Tensor | None = None, stream=None, wait=True,
                 objective_out: torch.Tensor | None = None, status_out: torch.Tensor | None = None,
                 stats=True, **opts):
    """dgs_solve_ex (stream-ordered): returns (status, sigma_out, objective,
    stats dict).  With wait (default) the stream is synchronised and status is
    the solve's outcome (dgs_stats.status); with wait=False a Pending whose
    result() does that.  objective_out / status_out: optional CUDA tensors
    (int64[1] / int32[1]) the device writes instead of host memory (the
    returned objective is then 0); stats=False passes no stats (the returned
    status is then the call's).

    Keyword options: init, init_sigma (int32 CUDA tensor), seed (random
    start), reeval (DGS_REEVAL_BOX / DGS_REEVAL_ALL), algorithm
    (DGS_ALG_PARALLEL / DGS_ALG_SEQUENTIAL), evaluation (DGS_EVAL_TILE_PAIRS /
    DGS_EVAL_ROW_OWNER), max_sweeps, deadline_us, profile (1: time the first
    evaluation and the greedy start; the call then waits), trace=(accepted
    int32, applied int32, objective int64) CUDA tensors of equal length."""
    n = _n(benefit)
    if sigma_out is None:
        sigma_out = torch.empty(n, dtype=torch.int32, device=benefit.device)
    o = _options(**opts)
    if status_out is not None:
        o.status_out = ctypes.c_void_p(status_out.data_ptr())
    f = ctypes.c_int64(0)
    fp = ctypes.c_void_p(objective_out.data_ptr()) if objective_out is not None else \
        ctypes.c_void_p(ctypes.addressof(f))
    s = dgs_stats()
    st = load().dgs_solve_ex(_dev(benefit, "benefit"), n, _dev(sigma_out, "sigma_out"), fp,
                             ctypes.byref(o), ctypes.byref(s) if stats else None, _stream(benefit, stream))
    pending = Pending(st, benefit, stream, sigma_out, f, s if stats else None, options=o, wait=wait)
    return pending.result() if wait else pending


def dgs_solve_rect(benefit: torch.Tensor, assign_out: torch.Tensor | None = None, stream=None, **opts):
    """dgs_solve_rect (stream-ordered; this wrapper waits): benefit is an
    n_agents x m_jobs int32 CUDA tensor; returns (status = the solve's
    outcome, assign_out (job or -1 per agent), objective, stats)."""
    if benefit.ndim != 2:
        raise ValueError("benefit must be an n_agents x m_jobs matrix")
    n, m = int(benefit.shape[0]), int(benefit.shape[1])
    if assign_out is None:
        assign_out = torch.empty(n, dtype=torch.int32, device=benefit.device)
    o = _options(**opts)
    f = ctypes.c_int64(0)
    s = dgs_stats()
    st = load().dgs_solve_rect(_dev(benefit, "benefit"), n, m, _dev(assign_out, "assign_out"), ctypes.byref(f),
                               ctypes.byref(o), ctypes.byref(s), _stream(benefit, stream))
    return Pending(st, benefit, stream, assign_out, f, s).result()


def dgs_solve_host(benefit: np.ndarray, stream=None, device=None, **opts):
    """dgs_solve_host: benefit is a host (numpy) int32 n x n array; returns
    (status, sigma_out numpy, objective, stats dict).  Copies are inside the call."""
    a = np.ascontiguousarray(benefit, dtype=np.int32)
    n = _n(a)
    out = np.empty(n, dtype=np.int32)
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    s_obj = stream if stream is not None else torch.cuda.current_stream(dev)
    o = _options(**opts)
    f = ctypes.c_int64(0)
    s = dgs_stats()
    st = load().dgs_solve_host(ctypes.c_void_p(a.ctypes.data), n, ctypes.c_void_p(out.ctypes.data),
                               ctypes.byref(f), ctypes.byref(o), ctypes.byref(s),
                               ctypes.c_void_p(s_obj.cuda_stream))
    return st, out, int(f.value), s.as_dict()


def dgs_evaluate(benefit: torch.Tensor, sigma_in: torch.Tensor, stream=None):
    """dgs_evaluate: returns (status, agent_gain, agent_job, job_gain, job_agent)."""
    n = _n(benefit)
    outs = [torch.empty(n, dtype=torch.int32, device=benefit.device) for _ in range(4)]
    st = load().dgs_evaluate(_dev(benefit, "benefit"), n, _dev(sigma_in, "sigma_in"),
                             *[_dev(o, "out") for o in outs], _stream(benefit, stream))
    return (st, *outs)


def dgs_evaluate_static(benefit: torch.Tensor, sigma_in: torch.Tensor, outputs=None, stream=None):
    """dgs_evaluate_static (no allocation inside the library): returns
    (status, agent_gain, agent_job, job_gain, job_agent).  ``outputs`` may hold
    four preallocated int32 CUDA tensors of length n."""
    n = _n(benefit)
    outs = outputs if outputs is not None else [torch.empty(n, dtype=torch.int32, device=benefit.device)
                                                for _ in range(4)]
    st = load().dgs_evaluate_static(_dev(benefit, "benefit"), n, _dev(sigma_in, "sigma_in"),
                                    *[_dev(o, "out") for o in outs], _stream(benefit, stream))
    return (st, *outs)


def dgs_greedy_init(benefit: torch.Tensor, sigma_out: torch.Tensor | None = None, stream=None):
    """dgs_greedy_init: returns (status, sigma_out)."""
    n = _n(benefit)
    if sigma_out is None:
        sigma_out = torch.empty(n, dtype=torch.int32, device=benefit.device)
    st = load().dgs_greedy_init(_dev(benefit, "benefit"), n, _dev(sigma_out, "sigma_out"),
                                _stream(benefit, stream))
    return st, sigma_out


def dgs_solve_batched(benefits, sigma_outs=None, stream=None, **opts):
    """dgs_solve_batched: ``benefits`` is a list of square int32 CUDA tensors
    (one device).  Returns (status, sigma_outs, objectives list, statuses
    list, stats dicts).  Keyword options as dgs_solve_ex (init, max_sweeps,
    deadline_us)."""
    count = len(benefits)
    if count == 0:
        raise ValueError("empty batch")
    ns = (ctypes.c_int32 * count)(*[_n(b) for b in benefits])
    if sigma_outs is None:
        sigma_outs = [torch.empty(_n(b), dtype=torch.int32, device=b.device) for b in benefits]
    a_ptrs = (ctypes.c_void_p * count)(*[_dev(b, "benefit").value for b in benefits])
    o_ptrs = (ctypes.c_void_p * count)(*[_dev(o, "sigma_out").value for o in sigma_outs])
    objs = (ctypes.c_int64 * count)()
    stats = (dgs_stats * count)()
    statuses = (ctypes.c_int * count)()
    o = _options(**opts)
    st = load().dgs_solve_batched(a_ptrs, ns, count, o_ptrs, objs, ctypes.byref(o), statuses, stats,
                                  _stream(benefits[0], stream))
    return st, sigma_outs, [int(x) for x in objs], [int(x) for x in statuses], [s.as_dict() for s in stats]


def dgs_server_request_bytes(n: int) -> int:
    return int(load().dgs_server_request_bytes(int(n)))


class Server:
    """dgs_server_* handle: create on the current CUDA device, submit host
    (numpy) or device (torch) matrices, poll or wait for tickets, destroy."""

    def __init__(self, budget_bytes: int, max_resident: int = 0):
        self._h = ctypes.c_void_p()
        self._keep = {}
        st = load().dgs_server_create(int(budget_bytes), int(max_resident), ctypes.byref(self._h))
        if st != DGS_OK:
            raise RuntimeError(f"dgs_server_create: {dgs_status_string(st)} {dgs_last_cuda_error()}")

    def dgs_submit(self, benefit):
        """Returns (status, ticket).  The matrix is kept referenced until its ticket is taken."""
        if isinstance(benefit, torch.Tensor):
            n, ptr, flags = _n(benefit), _dev(benefit, "benefit"), 0
        else:
            benefit = np.ascontiguousarray(benefit, dtype=np.int32)
            n, ptr, flags = _n(benefit), ctypes.c_void_p(benefit.ctypes.data), DGS_SUBMIT_HOST
        t = ctypes.c_uint64(0)
        st = load().dgs_submit(self._h, ptr, n, flags, ctypes.byref(t))
        if st == DGS_OK:
            self._keep[int(t.value)] = (benefit, n)
        return st, int(t.value)

    def dgs_submit_ex(self, benefit, init_sigma=None, **opts):
        """Returns (status, ticket).  init_sigma (numpy for host matrices, an
        int32 CUDA tensor for device ones) is a warm start; keyword options as
        dgs_solve_ex (init, seed, reeval, max_sweeps, deadline_us)."""
        if isinstance(benefit, torch.Tensor):
            n, ptr, flags = _n(benefit), _dev(benefit, "benefit"), 0
            o = _options(init_sigma=init_sigma, **opts)
        else:
            benefit = np.ascontiguousarray(benefit, dtype=np.int32)
            n, ptr, flags = _n(benefit), ctypes.c_void_p(benefit.ctypes.data), DGS_SUBMIT_HOST
            o = _options(**opts)
            if init_sigma is not None:
                init_sigma = np.ascontiguousarray(init_sigma, dtype=np.int32)
                o.init_sigma = ctypes.c_void_p(init_sigma.ctypes.data)
        if init_sigma is not None:
            o.init = DGS_INIT_USER
        t = ctypes.c_uint64(0)
        st = load().dgs_submit_ex(self._h, ptr, n, flags, ctypes.byref(o), ctypes.byref(t))
        if st == DGS_OK:
            self._keep[int(t.value)] = (benefit, n, init_sigma)
        return st, int(t.value)

    def _take(self, fn, ticket, *extra):
        n = self._keep[ticket][1] if ticket in self._keep else 0  # unknown: the library says so
        out = np.empty(max(n, 1), dtype=np.int32)
        f = ctypes.c_int64(0)
        s = dgs_stats()
        tm = dgs_request_times()
        st = fn(self._h, ctypes.c_uint64(ticket), *extra, ctypes.c_void_p(out.ctypes.data), ctypes.byref(f),
                ctypes.byref(s), ctypes.byref(tm))
        if st != DGS_PENDING:
            self._keep.pop(ticket, None)
        times = {k: getattr(tm, k) for k, _ in dgs_request_times._fields_}
        return st, out, int(f.value), s.as_dict(), times

    def dgs_poll(self, ticket: int):
        """Returns (status, sigma numpy, objective, stats, times); DGS_PENDING while running."""
        return self._take(load().dgs_poll, ticket)

    def dgs_server_wait(self, ticket: int, timeout_us: int = -1):
        return self._take(load().dgs_server_wait, ticket, ctypes.c_int64(int(timeout_us)))

    def dgs_cancel(self, ticket: int) -> int:
        return load().dgs_cancel(self._h, int(ticket))

    def dgs_server_get_info(self):
        info = dgs_server_info()
        st = load().dgs_server_get_info(self._h, ctypes.byref(info))
        return st, {name: (float if name.endswith("_ms") else int)(getattr(info, name)) for name, _ in info._fields_}

    def dgs_server_destroy(self):
        if self._h:
            load().dgs_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.dgs_server_destroy()

    def __del__(self):
        try:
            self.dgs_server_destroy()
        except Exception:
            pass


def dgs_server_create(budget_bytes: int, max_resident: int = 0) -> Server:
    return Server(budget_bytes, max_resident)


def dgs_autotune(n: int, stream=None, device=None):
    """dgs_autotune: returns (status, dict with the chosen shape, its size
    class and every candidate's time)."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    s_obj = stream if stream is not None else torch.cuda.current_stream(dev)
    r = dgs_tuning()
    st = load().dgs_autotune(int(n), ctypes.byref(r), ctypes.c_void_p(s_obj.cuda_stream))
    out = {"n_lo": r.n_lo, "n_hi": r.n_hi, "rows_per_thread": r.rows_per_thread, "strip": r.strip, "tma": r.tma,
           "best_ms": r.best_ms,
           "candidates": [{"rows_per_thread": r.cand_rows[k], "strip": r.cand_strip[k], "tma": r.cand_tma[k],
                           "ms": r.cand_ms[k]} for k in range(r.candidates)]}
    return st, out


def dgs_get_tuning(n: int):
    """Returns (status, rows_per_thread, strip, tma) used for solves of size n."""
    rows, strip, tma = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
    st = load().dgs_get_tuning(int(n), ctypes.byref(rows), ctypes.byref(strip), ctypes.byref(tma))
    return st, int(rows.value), int(strip.value), int(tma.value)


def dgs_read_bandwidth(buffer: torch.Tensor, repeats: int = 20, stream=None):
    """dgs_read_bandwidth on a contiguous CUDA tensor (its bytes, rounded down
    to a multiple of 16): returns (status, GB/s)."""
    if not (isinstance(buffer, torch.Tensor) and buffer.is_cuda and buffer.is_contiguous()):
        raise TypeError("buffer must be a contiguous CUDA tensor")
    nbytes = buffer.numel() * buffer.element_size() // 16 * 16
    gbs = ctypes.c_double(0.0)
    st = load().dgs_read_bandwidth(ctypes.c_void_p(buffer.data_ptr()), nbytes, int(repeats), ctypes.byref(gbs),
                                   _stream(buffer, stream))
    return st, float(gbs.value)


def dgs_release_cached_memory() -> int:
    """dgs_release_cached_memory: returns the status."""
    return int(load().dgs_release_cached_memory())
