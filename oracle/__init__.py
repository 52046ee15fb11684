"""CPU oracle for Deep Greedy Switching -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``dgs_oracle.c`` (plain,
C that follows Algorithms 2-4 of the paper, single-threaded unless
``set_evaluation`` asks otherwise, Section 3 and
Section 5) through ctypes.  It shares no code with the CUDA library.

Conventions: ``a`` is an n x n int32 numpy array, row = agent, column = job.
Assignments returned here are ``tau`` (agent -> job).

Functions without an independent pin: none -- every wrapped function is
pinned by the tests (hand traces, brute force, Hungarian bound, invariants).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dgs_oracle.c")
_HDR = os.path.join(_HERE, "dgs_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

INIT_GREEDY = 0
INIT_RANDOM = 1
INIT_IDENTITY = 2
INIT_USER = 3
CC_SLOTS = 0
CC_LITERAL_AGENTS = 1
REEVAL_BOX = 0
REEVAL_ALL = 1
OK = 0
ERR_INVALID = 1
ERR_RANGE = 2
TIMEOUT = 5


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC]
        )
        os.replace(tmp, _LIB)
    return _LIB


class _Stats(ctypes.Structure):
    _fields_ = [
        ("sweeps", ctypes.c_int32),
        ("passes", ctypes.c_int32),
        ("swaps_applied", ctypes.c_int64),
        ("evaluations", ctypes.c_int64),
    ]


_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    # DGS_ORACLE_LIB lets the mutation test load a deliberately broken copy.
    override = os.environ.get("DGS_ORACLE_LIB")
    lib = ctypes.CDLL(override if override else build())
    P = ctypes.c_void_p
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    lib.oracle_objective.argtypes = [P, i32, P]
    lib.oracle_objective.restype = i64
    lib.oracle_range_ok.argtypes = [P, i32]
    lib.oracle_range_ok.restype = ctypes.c_int
    lib.oracle_greedy_init.argtypes = [P, i32, P]
    lib.oracle_greedy_init.restype = None
    lib.oracle_ade.argtypes = [P, i32, P, P, i32, P, P]
    lib.oracle_ade.restype = None
    lib.oracle_jde.argtypes = [P, i32, P, P, i32, P, P]
    lib.oracle_jde.restype = None
    lib.oracle_evaluate_all.argtypes = [P, i32, P, P, P, P, P]
    lib.oracle_evaluate_all.restype = None
    lib.oracle_check_conflicts.argtypes = [i32, P, P, P, P, P, P, P]
    lib.oracle_check_conflicts.restype = None
    lib.oracle_dgs_parallel.argtypes = [P, i32, i32, P, ctypes.c_uint64, i32, i32, i32, P, P, P, i32, P, P, P]
    lib.oracle_random_permutation.argtypes = [i32, ctypes.c_uint64, P]
    lib.oracle_random_permutation.restype = None
    lib.oracle_splitmix64_next.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
    lib.oracle_splitmix64_next.restype = ctypes.c_uint64
    lib.oracle_dgs_parallel.restype = ctypes.c_int
    lib.oracle_dgs_sequential.argtypes = [P, i32, i32, P, ctypes.c_uint64, i32, P, P, P, i32, P, P, P, P, P, P]
    lib.oracle_dgs_sequential.restype = ctypes.c_int
    lib.oracle_dgs_rect.argtypes = [P, i32, i32, i32, i32, ctypes.c_uint64, i32, P, P, P]
    lib.oracle_dgs_rect.restype = ctypes.c_int
    lib.oracle_set_evaluation.argtypes = [i32, i32]
    lib.oracle_set_evaluation.restype = None
    lib.oracle_hungarian.argtypes = [P, i32, P]
    lib.oracle_hungarian.restype = i64
    lib.oracle_brute_force.argtypes = [P, i32, P]
    lib.oracle_brute_force.restype = i64
    _lib = lib
    return lib


def _c(arr: np.ndarray, dtype=np.int32) -> np.ndarray:
    return np.ascontiguousarray(arr, dtype=dtype)


def _p(arr: np.ndarray):
    return ctypes.c_void_p(arr.ctypes.data) if arr is not None else None


def objective(a, tau) -> int:
    a, tau = _c(a), _c(tau)
    return int(_load().oracle_objective(_p(a), a.shape[0], _p(tau)))


def range_ok(a) -> bool:
    a = _c(a)
    return bool(_load().oracle_range_ok(_p(a), a.shape[0]))


def greedy_init(a) -> np.ndarray:
    a = _c(a)
    tau = np.empty(a.shape[0], np.int32)
    _load().oracle_greedy_init(_p(a), a.shape[0], _p(tau))
    return tau


def ade(a, tau, i: int):
    """Algorithm 2 for agent i: (gain, job) -- (0, -1) when none improves."""
    a, tau = _c(a), _c(tau)
    sigma = np.empty_like(tau)
    sigma[tau] = np.arange(len(tau), dtype=np.int32)
    g, t = ctypes.c_int32(), ctypes.c_int32()
    _load().oracle_ade(_p(a), a.shape[0], _p(sigma), _p(tau), i, ctypes.byref(g), ctypes.byref(t))
    return g.value, t.value


def jde(a, tau, j: int):
    """JDE for job j: (gain, agent) -- (0, -1) when none improves."""
    a, tau = _c(a), _c(tau)
    sigma = np.empty_like(tau)
    sigma[tau] = np.arange(len(tau), dtype=np.int32)
    g, t = ctypes.c_int32(), ctypes.c_int32()
    _load().oracle_jde(_p(a), a.shape[0], _p(sigma), _p(tau), j, ctypes.byref(g), ctypes.byref(t))
    return g.value, t.value


def evaluate_all(a, tau):
    """Fresh evaluation of every slot: (agent_gain, agent_job, job_gain, job_agent)."""
    a, tau = _c(a), _c(tau)
    n = a.shape[0]
    out = [np.empty(n, np.int32) for _ in range(4)]
    _load().oracle_evaluate_all(_p(a), n, _p(tau), *[_p(o) for o in out])
    return tuple(out)


def check_conflicts(sigma, agent_gain, agent_job, job_gain, job_agent):
    """Algorithm 4 under reading R3: (in_ca, in_cj) as uint8 arrays."""
    sigma = _c(sigma)
    n = len(sigma)
    arrs = [_c(x) for x in (agent_gain, agent_job, job_gain, job_agent)]
    ca, cj = np.zeros(n, np.uint8), np.zeros(n, np.uint8)
    _load().oracle_check_conflicts(n, _p(sigma), *[_p(x) for x in arrs], _p(ca), _p(cj))
    return ca, cj


@dataclass
class SolveResult:
    status: int
    tau: np.ndarray
    objective: int
    sweeps: int
    passes: int
    swaps_applied: int
    evaluations: int
    trace_accepted: np.ndarray
    trace_applied: np.ndarray
    trace_objective: np.ndarray


def set_evaluation(threads: int = 1, transpose: bool = False) -> None:
    """Run Algorithm 3's slot evaluations on `threads` host threads, reading
    columns of a from a transposed copy when `transpose`.  Results do not
    depend on either; the default (1, False) is the literal loop."""
    _load().oracle_set_evaluation(int(threads), 1 if transpose else 0)


def random_permutation(n: int, seed: int) -> np.ndarray:
    """The random start: splitmix64 from seed, Fisher-Yates (Durstenfeld)."""
    tau = np.empty(max(n, 1), np.int32)
    _load().oracle_random_permutation(n, ctypes.c_uint64(seed), _p(tau))
    return tau[:n].copy()


def splitmix64(seed: int, count: int):
    """The first `count` outputs of splitmix64 started at seed."""
    state = ctypes.c_uint64(seed)
    return [int(_load().oracle_splitmix64_next(ctypes.byref(state))) for _ in range(count)]


def dgs_parallel(a, init: int = INIT_GREEDY, init_tau=None, max_sweeps: int = 0,
                 cc_rule: int = CC_SLOTS, trace_cap: int = 0, seed: int = 0,
                 reeval: int = REEVAL_BOX) -> SolveResult:
    """Algorithm 3 (parallel DGS) with the readings R1-R5 (reeval=REEVAL_ALL:
    every slot re-evaluated after each parallel switch; init=INIT_RANDOM:
    random start from seed)."""
    a = _c(a)
    n = a.shape[0]
    tau = np.zeros(max(n, 1), np.int32)
    f = ctypes.c_int64()
    st = _Stats()
    ta = np.zeros(max(trace_cap, 1), np.int32)
    tp = np.zeros(max(trace_cap, 1), np.int32)
    tf = np.zeros(max(trace_cap, 1), np.int64)
    it = _c(init_tau) if init_tau is not None else None
    status = _load().oracle_dgs_parallel(
        _p(a), n, init, _p(it), ctypes.c_uint64(seed), max_sweeps, cc_rule, reeval, _p(tau), ctypes.byref(f),
        ctypes.byref(st), trace_cap, _p(ta), _p(tp), _p(tf))
    k = min(st.sweeps, trace_cap)
    return SolveResult(status, tau[:n].copy(), f.value, st.sweeps, st.passes,
                       st.swaps_applied, st.evaluations, ta[:k].copy(), tp[:k].copy(), tf[:k].copy())


def dgs_sequential(a, init: int = INIT_GREEDY, init_tau=None, max_iters: int = 0, seed: int = 0,
                   trace_cap: int = 0) -> SolveResult:
    """Algorithm 1 (sequential DGS) with readings R1, R2, R5, R6.  ``sweeps``
    counts while-loop iterations; trace_applied holds 1 for each iteration
    that committed its exchange (trace_accepted is all ones)."""
    a = _c(a)
    n = a.shape[0]
    tau = np.zeros(max(n, 1), np.int32)
    f = ctypes.c_int64()
    st = _Stats()
    tp = np.zeros(max(trace_cap, 1), np.int32)
    tf = np.zeros(max(trace_cap, 1), np.int64)
    extra = [np.zeros(max(trace_cap, 1), np.int32) for _ in range(4)]
    it = _c(init_tau) if init_tau is not None else None
    status = _load().oracle_dgs_sequential(_p(a), n, init, _p(it), ctypes.c_uint64(seed), max_iters, _p(tau),
                                           ctypes.byref(f), ctypes.byref(st), trace_cap, _p(tp), _p(tf),
                                           *[_p(x) for x in extra])
    k = min(st.sweeps, trace_cap)
    r = SolveResult(status, tau[:n].copy(), f.value, st.sweeps, st.passes, st.swaps_applied, st.evaluations,
                    np.ones(k, np.int32), tp[:k].copy(), tf[:k].copy())
    r.trace_slot, r.trace_target, r.trace_u, r.trace_v = (x[:k].copy() for x in extra)
    return r


def dgs_rect(a, algorithm: int = 0, init: int = INIT_GREEDY, seed: int = 0, reeval: int = REEVAL_BOX):
    """Rectangular instance (n agents x m jobs): (status, assignment with -1
    for agents left on a dummy job, objective, sweeps)."""
    a = _c(a)
    n, m = a.shape
    out = np.empty(n, np.int32)
    f = ctypes.c_int64()
    st = _Stats()
    status = _load().oracle_dgs_rect(_p(a), n, m, algorithm, init, ctypes.c_uint64(seed), reeval, _p(out),
                                     ctypes.byref(f), ctypes.byref(st))
    return status, out, f.value, st.sweeps


def hungarian(a):
    """Exact maximum (value, tau) by the Hungarian method."""
    a = _c(a)
    tau = np.empty(a.shape[0], np.int32)
    v = _load().oracle_hungarian(_p(a), a.shape[0], _p(tau))
    return int(v), tau


def brute_force(a):
    """Exact maximum (value, tau) by enumerating permutations (n <= 10)."""
    a = _c(a)
    tau = np.empty(a.shape[0], np.int32)
    v = _load().oracle_brute_force(_p(a), a.shape[0], _p(tau))
    return int(v), tau
