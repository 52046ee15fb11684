"""GPU path (C ABI, sm_103a kernels) against the CPU oracle, element by element.

Integer work throughout, so the bar is bit-exactness: assignment, objective,
sweep count, per-sweep trace and every slot of a fresh evaluation.
"""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1106_5694_gb300 import binding as B
from paper_1106_5694_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_traces.json")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1106_5694_gb300 import build_ext
    build_ext.build()
    oracle.build()
    B.load()


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def _make(kind, n, seed):
    if kind == "uniform":
        return inputs.uniform(n, 0, 1000, seed)
    if kind == "wide":
        return inputs.uniform(n, -(10**8), 10**8, seed)
    if kind == "peer":
        return inputs.peer_shaped(n, seed)
    if kind == "ties":
        return inputs.uniform(n, 0, 4, seed)
    if kind == "geom":
        return inputs.geom(n, 1000.0, seed)
    if kind == "constant":
        return np.full((n, n), 5, np.int32)
    raise ValueError(kind)


# ------------------------------------------------------- difference evaluation
EVAL_CASES = [(k, n, s) for k in ("uniform", "ties", "peer", "wide")
              for n in (1, 2, 3, 5, 63, 64, 65, 130, 257, 301) for s in (0, 1)]


@pytest.mark.parametrize("kind,n,seed", EVAL_CASES)
def test_evaluate_matches_oracle(kind, n, seed):
    a = _make(kind, n, seed)
    tau = inputs.random_permutation(n, 1000 + seed)
    st, ag, aj, jg, ja = B.dgs_evaluate(_cuda(a), _cuda(tau))
    assert st == B.DGS_OK, B.dgs_status_string(st)
    want = oracle.evaluate_all(a, tau)
    for got, exp, name in zip((ag, aj, jg, ja), want, ("agent_gain", "agent_job", "job_gain", "job_agent")):
        np.testing.assert_array_equal(got.cpu().numpy(), exp, err_msg=name)


# --------------------------------------------------------------- greedy start
GREEDY_CASES = [(k, n, s) for k in ("uniform", "ties", "peer", "constant")
                for n in (1, 7, 64, 100, 256, 513) for s in (0, 1)]


@pytest.mark.parametrize("kind,n,seed", GREEDY_CASES)
def test_greedy_matches_oracle(kind, n, seed):
    a = _make(kind, n, seed)
    st, sig = B.dgs_greedy_init(_cuda(a))
    assert st == B.DGS_OK
    np.testing.assert_array_equal(sig.cpu().numpy(), oracle.greedy_init(a))


@pytest.mark.parametrize("kind,n,seed", [("ties", 300, 1), ("peer", 2000, 2), ("uniform", 1500, 3), ("wide", 97, 4)])
def test_greedy_rounds_fallback_equals_deferred_acceptance(kind, n, seed, monkeypatch):
    """The fallback greedy start (locally-dominant rounds run as a device
    loop) and deferred acceptance give the same assignment, the oracle's."""
    a = _make(kind, n, seed)
    ref = oracle.greedy_init(a)
    st, sig = B.dgs_greedy_init(_cuda(a))
    assert st == B.DGS_OK
    np.testing.assert_array_equal(sig.cpu().numpy(), ref)
    monkeypatch.setenv("DGS_GREEDY_ROUNDS", "1")
    st, sig_r = B.dgs_greedy_init(_cuda(a))
    assert st == B.DGS_OK
    np.testing.assert_array_equal(sig_r.cpu().numpy(), ref)
    st, tau, f, stats = B.dgs_solve_ex(_cuda(a))
    full = oracle.dgs_parallel(a)
    assert st == B.DGS_OK and f == full.objective and stats["sweeps"] == full.sweeps
    np.testing.assert_array_equal(tau.cpu().numpy(), full.tau)


_FF_REF = {}


@pytest.mark.parametrize("colour", ["0", "1"])
@pytest.mark.parametrize("kind,n,seed", [("uniform", 1500, 3), ("wide", 1500, 5), ("ties", 700, 1), ("peer", 1200, 2),
                                         ("wide", 300, 6)])
def test_colouring_pass_matches_oracle(kind, n, seed, colour, monkeypatch):
    """Runs of quiet sweeps taken by colouring passes (DGS_CC_COLOUR=1, the
    default) or one sweep at a time (0): the same sweeps, per-sweep accepted
    counts and objectives, and assignment as the oracle.  The wide-range
    inputs give long quiet runs with many passes; n = 300 runs in the
    single-CTA loop."""
    a = _make(kind, n, seed)
    key = (kind, n, seed)
    if key not in _FF_REF:
        _FF_REF[key] = oracle.dgs_parallel(a, trace_cap=100000)
    ref = _FF_REF[key]
    monkeypatch.setenv("DGS_CC_COLOUR", colour)
    tr = _trace_tensors(max(ref.sweeps, 1))
    st, sig, f, stats = B.dgs_solve_ex(_cuda(a), trace=tr)
    assert st == B.DGS_OK, B.dgs_status_string(st)
    np.testing.assert_array_equal(sig.cpu().numpy(), ref.tau)
    assert f == ref.objective and stats["sweeps"] == ref.sweeps
    k = ref.sweeps
    np.testing.assert_array_equal(tr[0][:k].cpu().numpy(), ref.trace_accepted)
    np.testing.assert_array_equal(tr[1][:k].cpu().numpy(), ref.trace_applied)
    np.testing.assert_array_equal(tr[2][:k].cpu().numpy(), ref.trace_objective)


@pytest.mark.parametrize("cap", [1, 3, 9, 40, 200])
def test_colouring_pass_stops_at_the_sweep_cap(cap):
    """A pass never runs past the sweep cap: the capped solve is the oracle's
    prefix on a long quiet run."""
    a = _make("wide", 1000, 8)
    ref = oracle.dgs_parallel(a, max_sweeps=cap)
    st, sig, f, stats = B.dgs_solve_ex(_cuda(a), max_sweeps=cap)
    assert st == (B.DGS_TIMEOUT if ref.status == oracle.TIMEOUT else B.DGS_OK)
    np.testing.assert_array_equal(sig.cpu().numpy(), ref.tau)
    assert f == ref.objective and stats["sweeps"] == ref.sweeps


# ------------------------------------------------------------------ full solve
SOLVE_CASES = [(k, n, s) for k in ("uniform", "ties", "peer", "geom", "wide")
               for n in (2, 3, 9, 33, 64, 129, 200) for s in (0, 1)] + \
              [("uniform", 512, 0), ("peer", 512, 1), ("ties", 401, 2), ("uniform", 1024, 3), ("peer", 1024, 0)]


def _trace_tensors(cap):
    return (torch.zeros(cap, dtype=torch.int32, device="cuda"), torch.zeros(cap, dtype=torch.int32, device="cuda"),
            torch.zeros(cap, dtype=torch.int64, device="cuda"))


@pytest.mark.parametrize("kind,n,seed", SOLVE_CASES)
def test_solve_matches_oracle(kind, n, seed):
    a = _make(kind, n, seed)
    ref = oracle.dgs_parallel(a, trace_cap=100000)
    assert ref.status == oracle.OK
    tr = _trace_tensors(max(ref.sweeps, 1))
    st, sig, f, stats = B.dgs_solve_ex(_cuda(a), trace=tr)
    assert st == B.DGS_OK, B.dgs_status_string(st)
    np.testing.assert_array_equal(sig.cpu().numpy(), ref.tau)
    assert f == ref.objective
    assert stats["sweeps"] == ref.sweeps
    assert stats["swaps_applied"] == ref.swaps_applied
    k = ref.sweeps
    np.testing.assert_array_equal(tr[0][:k].cpu().numpy(), ref.trace_accepted)
    np.testing.assert_array_equal(tr[1][:k].cpu().numpy(), ref.trace_applied)
    np.testing.assert_array_equal(tr[2][:k].cpu().numpy(), ref.trace_objective)


@pytest.mark.parametrize("name", ["n3_identity", "n2_antidiagonal"])
def test_hand_traces_on_gpu(name):
    with open(GOLDEN) as fh:
        t = {x["name"]: x for x in json.load(fh)["traces"]}[name]
    a = np.array(t["a"], np.int32)
    tr = _trace_tensors(16)
    st, sig, f, stats = B.dgs_solve_ex(_cuda(a), init=B.DGS_INIT_IDENTITY, trace=tr)
    assert st == B.DGS_OK
    assert sig.cpu().tolist() == t["tau"] and f == t["objective"] and stats["sweeps"] == t["sweeps"]
    k = t["sweeps"]
    assert tr[0][:k].cpu().tolist() == t["accepted"]
    assert tr[1][:k].cpu().tolist() == t["applied"]


@pytest.mark.parametrize("init", ["identity", "user"])
@pytest.mark.parametrize("kind,n,seed", [("uniform", 150, 4), ("peer", 97, 5), ("ties", 64, 6)])
def test_other_starts_match_oracle(init, kind, n, seed):
    a = _make(kind, n, seed)
    if init == "identity":
        ref = oracle.dgs_parallel(a, init=oracle.INIT_IDENTITY)
        st, sig, f, stats = B.dgs_solve_ex(_cuda(a), init=B.DGS_INIT_IDENTITY)
    else:
        p = inputs.random_permutation(n, seed)
        ref = oracle.dgs_parallel(a, init=oracle.INIT_USER, init_tau=p)
        st, sig, f, stats = B.dgs_solve_ex(_cuda(a), init=B.DGS_INIT_USER, init_sigma=_cuda(p))
    assert st == B.DGS_OK
    np.testing.assert_array_equal(sig.cpu().numpy(), ref.tau)
    assert f == ref.objective and stats["sweeps"] == ref.sweeps


@pytest.mark.parametrize("cap", [1, 2, 5, 17])
def test_sweep_cap_matches_oracle_prefix(cap):
    a = _make("uniform", 300, 9)
    ref = oracle.dgs_parallel(a, max_sweeps=cap)
    st, sig, f, stats = B.dgs_solve_ex(_cuda(a), max_sweeps=cap)
    expect = B.DGS_TIMEOUT if ref.status == oracle.TIMEOUT else B.DGS_OK
    assert st == expect
    np.testing.assert_array_equal(sig.cpu().numpy(), ref.tau)
    assert f == ref.objective and stats["sweeps"] == ref.sweeps


def test_unwaited_solves_keep_their_host_outputs():
    """Solves enqueued with wait=False and their Pending dropped at once: the
    host memory their stream callbacks write (objective, stats) stays alive
    until the stream gets there, and later results are right."""
    import ctypes
    import gc

    a = _make("peer", 256, 3)
    at = _cuda(a)
    ref = oracle.dgs_parallel(a)
    sig = torch.empty(256, dtype=torch.int32, device="cuda")
    for k in range(120):
        B.dgs_solve_ex(at, sigma_out=sig, wait=False, stats=(k % 2 == 0))
        B.dgs_solve(at, sigma_out=sig, wait=False)
        junk = [ctypes.c_int64(-1) for _ in range(64)]  # take over freed host memory
        del junk
        if k % 16 == 0:
            gc.collect()
    torch.cuda.synchronize()
    st, tau, f, stats = B.dgs_solve_ex(at, wait=False).result()
    assert st == B.DGS_OK and f == ref.objective and stats["sweeps"] == ref.sweeps
    np.testing.assert_array_equal(tau.cpu().numpy(), ref.tau)
    st, tau, f = B.dgs_solve(at, wait=False).result()
    assert st == B.DGS_OK and f == ref.objective


def test_errors():
    a = _make("uniform", 20, 0)
    bad = a.copy()
    bad[3, 4] = 1 << 29
    # stream-ordered: the call is accepted, the outcome arrives with the stream
    st, sig, _ = B.dgs_solve(_cuda(bad))
    assert st == B.DGS_OK and bool((sig == -1).all())
    assert B.dgs_solve_ex(_cuda(bad))[0] == B.DGS_ERR_RANGE
    neg = a.copy()
    neg[0, 0] = -(1 << 29)
    assert B.dgs_solve_ex(_cuda(neg))[0] == B.DGS_ERR_RANGE
    # the outcome also lands in a device word (options.status_out)
    word = torch.full((1,), -5, dtype=torch.int32, device="cuda")
    st, sig, _, stats = B.dgs_solve_ex(_cuda(neg), status_out=word)
    assert st == stats["status"] == B.DGS_ERR_RANGE and int(word.item()) == B.DGS_ERR_RANGE
    dup = np.arange(20, dtype=np.int32)
    dup[5] = 6
    st, _, _, _ = B.dgs_solve_ex(_cuda(a), init=B.DGS_INIT_USER, init_sigma=_cuda(dup))
    assert st == B.DGS_ERR_INVALID
    empty = torch.zeros((0, 0), dtype=torch.int32, device="cuda")
    assert B.dgs_solve(empty)[0] == B.DGS_ERR_INVALID
    # library stays usable after errors
    st, sig, f = B.dgs_solve(_cuda(a))
    assert st == B.DGS_OK and f == oracle.dgs_parallel(a).objective


def test_single_agent():
    st, sig, f = B.dgs_solve(_cuda(np.array([[-7]], np.int32)))
    assert st == B.DGS_OK and sig.cpu().tolist() == [0] and f == -7


def test_host_entry_point_matches_device():
    a = _make("peer", 210, 3)
    st_h, sig_h, f_h, _ = B.dgs_solve_host(a)
    st_d, sig_d, f_d = B.dgs_solve(_cuda(a))
    assert st_h == st_d == B.DGS_OK
    np.testing.assert_array_equal(sig_h, sig_d.cpu().numpy())
    assert f_h == f_d


@pytest.mark.parametrize("kind,n,init", [("peer", 2048, "greedy"), ("uniform", 2500, "greedy"),
                                         ("peer", 2052, "greedy"), ("peer", 2050, "greedy"),
                                         ("uniform", 2100, "random"), ("ties", 4096, "greedy")])
def test_host_entry_point_in_bands_matches_device(kind, n, init):
    """dgs_solve_host copies a large matrix in row bands on a copy stream and
    starts greedy pass 1 on each band as it lands (n a multiple of 4, greedy
    start; otherwise one copy): the result equals the device-resident solve."""
    a = _make(kind, n, 5)
    opts = {} if init == "greedy" else {"init": B.DGS_INIT_RANDOM, "seed": 7}
    st_h, sig_h, f_h, stats_h = B.dgs_solve_host(a, **opts)
    st_d, sig_d, f_d, stats_d = B.dgs_solve_ex(_cuda(a), **opts)
    assert st_h == st_d == B.DGS_OK
    np.testing.assert_array_equal(sig_h, sig_d.cpu().numpy())
    assert f_h == f_d and stats_h["sweeps"] == stats_d["sweeps"]


def test_deterministic_repeat():
    a = _make("uniform", 700, 11)
    outs = [B.dgs_solve(_cuda(a)) for _ in range(3)]
    for st, sig, f in outs:
        assert st == B.DGS_OK and f == outs[0][2]
        assert torch.equal(sig, outs[0][1])


# ------------------------------------------ larger sizes: prefix + properties
def _local_opt_gpu(a_t, sig):
    n = a_t.shape[0]
    a64 = a_t.to(torch.int64)
    d = a64[torch.arange(n, device="cuda"), sig.long()]
    cross = a64[:, sig.long()]
    g = cross + cross.T - d[:, None] - d[None, :]
    return int(g.max().item())


@pytest.mark.parametrize("kind,n", [("peer", 4096), ("uniform", 4096)])
def test_workload_4096_prefix_and_properties(kind, n):
    a = inputs.peer_shaped(n, 0) if kind == "peer" else inputs.uniform(n, 0, 10**6, 0)
    at = _cuda(a)
    # exact prefix: the first sweeps equal the oracle's
    cap = 3
    ref = oracle.dgs_parallel(a, max_sweeps=cap, trace_cap=cap)
    tr = _trace_tensors(cap)
    st, sig, f, stats = B.dgs_solve_ex(at, max_sweeps=cap, trace=tr)
    assert st == (B.DGS_TIMEOUT if ref.status == oracle.TIMEOUT else B.DGS_OK)
    np.testing.assert_array_equal(sig.cpu().numpy(), ref.tau)
    assert f == ref.objective
    np.testing.assert_array_equal(tr[0][:ref.sweeps].cpu().numpy(), ref.trace_accepted)
    # full solve: permutation, exact objective, no improving 2-exchange
    st, sig, f, stats = B.dgs_solve_ex(at)
    assert st == B.DGS_OK
    s = sig.cpu().numpy()
    assert np.array_equal(np.sort(s), np.arange(n))
    assert f == int(a[np.arange(n), s].astype(np.int64).sum())
    assert _local_opt_gpu(at, sig) <= 0
    assert f >= stats["initial_objective"]


# ------------------------------- every internal path gives the same result
_KNOB_SCRIPT = r"""
import sys, json, numpy as np, torch
sys.path.insert(0, {root!r})
from paper_1106_5694_gb300 import binding as B, inputs
out = []
for kind, n, seed in {cases!r}:
    a = inputs.peer_shaped(n, seed) if kind == "peer" else \
        inputs.uniform(n, -(10**8), 10**8, seed) if kind == "wide" else inputs.uniform(n, 0, 1000, seed)
    st, sig, f, stats = B.dgs_solve_ex(torch.from_numpy(a).cuda(), evaluation={evaluation!r})
    out.append([st, f, stats["sweeps"], sig.cpu().tolist()])
print(json.dumps(out))
"""


def _run_knob_cases(env, evaluation=0, cases=None):
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cases = cases or [("uniform", 300, 1), ("peer", 257, 2), ("uniform", 513, 3), ("peer", 640, 4)]
    code = _KNOB_SCRIPT.format(root=root, cases=cases, evaluation=evaluation)
    r = subprocess.run([sys.executable, "-c", code], env=dict(os.environ, **env), capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr
    got = json.loads(r.stdout.strip().splitlines()[-1])
    for (kind, n, seed), (st, f, sweeps, tau) in zip(cases, got):
        a = _make(kind, n, seed)
        ref = oracle.dgs_parallel(a)
        assert st == B.DGS_OK and f == ref.objective and sweeps == ref.sweeps
        assert tau == ref.tau.tolist()


@pytest.mark.parametrize("env", [{"DGS_UPDATE_POLICY": "1"}, {"DGS_UPDATE_POLICY": "2"},
                                 {"DGS_CTL_MODE": "1"}, {"DGS_CTL_MODE": "0"},
                                 {"DGS_CTL_MODE": "0", "DGS_UPDATE_POLICY": "2"},
                                 {"DGS_SHORT_WRAPS": "1"}, {"DGS_SHORT_WRAPS": "1", "DGS_CTL_MODE": "1"},
                                 {"DGS_EXACT_KEYS": "1"}, {"DGS_EVAL_ROWS": "8"},
                                 {"DGS_EVAL_ROWS": "8", "DGS_EXACT_KEYS": "1", "DGS_UPDATE_POLICY": "1"},
                                 {"DGS_EVAL_ROWS": "4", "DGS_EVAL_STRIP": "3", "DGS_UPDATE_POLICY": "1"},
                                 {"DGS_EVAL_STRIP": "1", "DGS_EXACT_KEYS": "1", "DGS_UPDATE_POLICY": "1"},
                                 {"DGS_EVAL_STRIP": "32", "DGS_UPDATE_POLICY": "1"},
                                 {"DGS_EVAL_STRIP": "0", "DGS_UPDATE_POLICY": "1"},
                                 {"DGS_EVAL_STRIP": "0", "DGS_EVAL_ROWS": "4", "DGS_EXACT_KEYS": "1"},
                                 {"DGS_EVAL_TMA": "1", "DGS_EVAL_STRIP": "0", "DGS_UPDATE_POLICY": "1"},
                                 {"DGS_EVAL_TMA": "1", "DGS_EVAL_STRIP": "8", "DGS_EVAL_ROWS": "4",
                                  "DGS_UPDATE_POLICY": "1"},
                                 {"DGS_EVAL_TMA": "1", "DGS_EXACT_KEYS": "1", "DGS_UPDATE_POLICY": "1"},
                                 {"DGS_EVAL_ROWS": "16", "DGS_EVAL_STRIP": "0", "DGS_UPDATE_POLICY": "1"},
                                 {"DGS_EVAL_ROWS": "16", "DGS_EVAL_STRIP": "3", "DGS_EXACT_KEYS": "1",
                                  "DGS_UPDATE_POLICY": "1"},
                                 {"DGS_EVAL_ROWS": "16", "DGS_EVAL_STRIP": "32"},
                                 {"DGS_CTL_COMPACT_MIN": "1"}, {"DGS_CTL_COMPACT_MIN": "1", "DGS_CTL_MODE": "0"},
                                 {"DGS_CTL_COMPACT_MIN": "1", "DGS_SHORT_WRAPS": "1"},
                                 {"DGS_CTL_COMPACT_MIN": "1", "DGS_CTL_MODE": "1"},
                                 {"DGS_CTL_COMPACT_MIN": "1", "DGS_CTL_MODE": "1", "DGS_SHORT_WRAPS": "1"}])
def test_internal_paths_agree_with_oracle(env):
    """Forcing the full-evaluation or row-task update path, placing the
    controller's scratch in global memory, making its reservation keys and
    claim stamps wrap every few rounds, compacting its edge list at every
    chance, disabling the evaluation kernel's packed 32-bit keys, or running
    it with other launch shapes (rows per thread, strip length, TMA gathers),
    must not change any result."""
    _run_knob_cases(env)


@pytest.mark.parametrize("env", [{"DGS_SHORT_WRAPS": "1"}, {"DGS_SHORT_WRAPS": "1", "DGS_CTL_COMPACT_MIN": "1"},
                                 {"DGS_SMALL_LOOP_THREADS": "256"}, {"DGS_SMALL_LOOP_THREADS": "1024"},
                                 {"DGS_CTL_MODE": "1"}, {"DGS_CTL_MODE": "1", "DGS_CTL_COMPACT_MIN": "1"}])
def test_colouring_passes_under_knobs_agree_with_oracle(env):
    """Long quiet runs (wide-range values; the single-CTA loop at n = 700, the
    graph loop at n = 1300) under reservation keys and claim stamps that wrap
    every few rounds, compaction at every chance, or other widths of the
    single-CTA loop: the oracle's results."""
    _run_knob_cases(env, cases=[("wide", 700, 7), ("wide", 1300, 8)])


# ------------------------- the row-owner (A-transpose) evaluation kernel
ROW_OWNER_CASES = [(k, n, 0) for k in ("uniform", "ties", "peer", "wide") for n in (1, 2, 3, 5, 63, 65, 130, 257)] + \
                  [("peer", 1000, 1), ("uniform", 777, 2), ("geom", 300, 3)]


@pytest.mark.parametrize("kind,n,seed", ROW_OWNER_CASES)
def test_row_owner_evaluation_matches_oracle(kind, n, seed):
    """Every full evaluation by the row-owner kernel: the solve, its trace and
    its sweep count equal the oracle's."""
    a = _make(kind, n, seed)
    ref = oracle.dgs_parallel(a, trace_cap=100000)
    tr = _trace_tensors(max(ref.sweeps, 1))
    st, sig, f, stats = B.dgs_solve_ex(_cuda(a), trace=tr, evaluation=B.DGS_EVAL_ROW_OWNER)
    assert st == B.DGS_OK, B.dgs_status_string(st)
    np.testing.assert_array_equal(sig.cpu().numpy(), ref.tau)
    assert f == ref.objective and stats["sweeps"] == ref.sweeps and stats["swaps_applied"] == ref.swaps_applied
    k = ref.sweeps
    np.testing.assert_array_equal(tr[0][:k].cpu().numpy(), ref.trace_accepted)
    np.testing.assert_array_equal(tr[2][:k].cpu().numpy(), ref.trace_objective)


def test_row_owner_evaluation_other_starts_rules_and_sequential():
    a = _make("peer", 200, 9)
    for kw, okw in (({"init": B.DGS_INIT_RANDOM, "seed": 5}, {"init": oracle.INIT_RANDOM, "seed": 5}),
                    ({"reeval": B.DGS_REEVAL_ALL}, {"reeval": oracle.REEVAL_ALL})):
        ref = oracle.dgs_parallel(a, **okw)
        st, sig, f, stats = B.dgs_solve_ex(_cuda(a), evaluation=B.DGS_EVAL_ROW_OWNER, **kw)
        assert st == B.DGS_OK
        np.testing.assert_array_equal(sig.cpu().numpy(), ref.tau)
        assert f == ref.objective and stats["sweeps"] == ref.sweeps
    ref = oracle.dgs_sequential(a)
    st, sig, f, stats = B.dgs_solve_ex(_cuda(a), algorithm=B.DGS_ALG_SEQUENTIAL, evaluation=B.DGS_EVAL_ROW_OWNER)
    assert st == B.DGS_OK
    np.testing.assert_array_equal(sig.cpu().numpy(), ref.tau)
    assert f == ref.objective


@pytest.mark.parametrize("env", [{"DGS_UPDATE_POLICY": "1"}, {"DGS_UPDATE_POLICY": "1", "DGS_CTL_MODE": "0"}, {}])
def test_row_owner_evaluation_update_paths_agree_with_oracle(env):
    """The row-owner kernel also runs the conditional full re-evaluations
    (forced after every commit by DGS_UPDATE_POLICY=1)."""
    _run_knob_cases(env, evaluation=B.DGS_EVAL_ROW_OWNER)


def _best_exchange_gain_blocked(at, sig, block=2048):
    """max over agent pairs of the 2-exchange gain (row blocks, int64)."""
    n = at.shape[0]
    s64 = sig.long()
    d = at[torch.arange(n, device=at.device), s64].long()
    best = -(1 << 62)
    for r0 in range(0, n, block):
        cross = at[r0:r0 + block][:, s64].long()
        back = at[:, s64[r0:r0 + block]].long().T
        g = cross + back - d[r0:r0 + block, None] - d[None, :]
        best = max(best, int(g.max().item()))
    return best


def test_row_owner_unstaged_rows_agree_with_tile_pairs():
    """n = 28000: a row of the transpose is too long for two shared-memory
    stages, so the row-owner kernel gathers it from global memory.  The solve
    equals the tile-pair solve (itself bit-exact with the oracle at every size
    the oracle reaches) and is a 2-exchange local optimum with its exact
    objective."""
    n = 28000
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    at = torch.randint(0, 10**6, (n, n), dtype=torch.int32, device="cuda", generator=g)
    st1, sig1, f1, s1 = B.dgs_solve_ex(at)
    st2, sig2, f2, s2 = B.dgs_solve_ex(at, evaluation=B.DGS_EVAL_ROW_OWNER)
    assert st1 == B.DGS_OK and st2 == B.DGS_OK
    assert torch.equal(sig1, sig2) and f1 == f2 and s1["sweeps"] == s2["sweeps"]
    assert torch.equal(torch.sort(sig2.long()).values, torch.arange(n, device="cuda"))
    assert f2 == int(at[torch.arange(n, device="cuda"), sig2.long()].long().sum().item())
    assert _best_exchange_gain_blocked(at, sig2) <= 0
    del at
    torch.cuda.empty_cache()


# ------------------- the paper's random start and the re-evaluate-all rule
RULE_CASES = [(k, n, s) for k in ("uniform", "peer", "geom", "ties") for n in (2, 9, 64, 129, 300) for s in (0, 1)]


@pytest.mark.parametrize("kind,n,seed", RULE_CASES)
def test_random_start_and_reeval_rules_match_oracle(kind, n, seed):
    a = _make(kind, n, seed)
    for init, reeval in ((oracle.INIT_RANDOM, oracle.REEVAL_BOX), (oracle.INIT_RANDOM, oracle.REEVAL_ALL),
                         (oracle.INIT_GREEDY, oracle.REEVAL_ALL)):
        ref = oracle.dgs_parallel(a, init=init, seed=1000 + seed, reeval=reeval, trace_cap=100000)
        assert ref.status == oracle.OK
        tr = _trace_tensors(max(ref.sweeps, 1))
        st, sig, f, stats = B.dgs_solve_ex(_cuda(a), init=init, seed=1000 + seed, reeval=reeval, trace=tr)
        assert st == B.DGS_OK, B.dgs_status_string(st)
        np.testing.assert_array_equal(sig.cpu().numpy(), ref.tau)
        assert f == ref.objective and stats["sweeps"] == ref.sweeps and stats["swaps_applied"] == ref.swaps_applied
        k = ref.sweeps
        np.testing.assert_array_equal(tr[0][:k].cpu().numpy(), ref.trace_accepted)
        np.testing.assert_array_equal(tr[1][:k].cpu().numpy(), ref.trace_applied)


def test_hand_trace_reeval_all_on_gpu():
    with open(GOLDEN) as fh:
        t = {x["name"]: x for x in json.load(fh)["traces"]}["n3_identity_reeval_all"]
    tr = _trace_tensors(4)
    st, sig, f, stats = B.dgs_solve_ex(_cuda(np.array(t["a"], np.int32)), init=B.DGS_INIT_IDENTITY,
                                       reeval=B.DGS_REEVAL_ALL, trace=tr)
    assert st == B.DGS_OK
    assert sig.cpu().tolist() == t["tau"] and f == t["objective"] and stats["sweeps"] == t["sweeps"]
    assert tr[0][:1].cpu().tolist() == t["accepted"] and tr[1][:1].cpu().tolist() == t["applied"]


def test_batched_random_start_and_reeval_all_match_oracle():
    cases = [("geom", 150, 3), ("peer", 97, 5), ("uniform", 301, 6), ("ties", 64, 7), ("geom", 40, 8)]
    mats = [_make(*c) for c in cases]
    for reeval in (B.DGS_REEVAL_BOX, B.DGS_REEVAL_ALL):
        st, sigs, objs, sts, stats = B.dgs_solve_batched([_cuda(a) for a in mats], init=B.DGS_INIT_RANDOM, seed=77,
                                                         reeval=reeval)
        assert st == B.DGS_OK, B.dgs_last_cuda_error()
        for a, sig, f, s in zip(mats, sigs, objs, stats):
            ref = oracle.dgs_parallel(a, init=oracle.INIT_RANDOM, seed=77, reeval=reeval)
            np.testing.assert_array_equal(sig.cpu().numpy(), ref.tau)
            assert f == ref.objective and s["sweeps"] == ref.sweeps


def test_invalid_rule_and_start_rejected():
    a = _cuda(_make("uniform", 20, 0))
    assert B.dgs_solve_ex(a, reeval=7)[0] == B.DGS_ERR_INVALID
    assert B.dgs_solve_ex(a, init=9)[0] == B.DGS_ERR_INVALID
    assert B.dgs_solve_ex(a, evaluation=2)[0] == B.DGS_ERR_INVALID
    assert B.dgs_solve_batched([a], evaluation=B.DGS_EVAL_ROW_OWNER)[0] == B.DGS_ERR_INVALID


# --------------------------------------------- Algorithm 1 (sequential DGS)
SEQ_CASES = [(k, n, s) for k in ("uniform", "peer", "ties", "geom", "wide") for n in (2, 3, 9, 64, 130, 257) for s in (0, 1)] + \
            [("peer", 1000, 2), ("uniform", 700, 3), ("peer", 6500, 4)]


@pytest.mark.parametrize("kind,n,seed", SEQ_CASES)
def test_sequential_matches_oracle(kind, n, seed):
    a = _make(kind, n, seed)
    for init in (oracle.INIT_GREEDY, oracle.INIT_RANDOM):
        ref = oracle.dgs_sequential(a, init=init, seed=seed, trace_cap=1 << 20)
        assert ref.status == oracle.OK
        tr = _trace_tensors(max(ref.sweeps, 1))
        st, sig, f, stats = B.dgs_solve_ex(_cuda(a), init=init, seed=seed, algorithm=B.DGS_ALG_SEQUENTIAL, trace=tr)
        assert st == B.DGS_OK, (B.dgs_status_string(st), B.dgs_last_cuda_error())
        np.testing.assert_array_equal(sig.cpu().numpy(), ref.tau)
        assert f == ref.objective and stats["sweeps"] == ref.sweeps and stats["swaps_applied"] == ref.swaps_applied
        k = ref.sweeps
        np.testing.assert_array_equal(tr[1][:k].cpu().numpy(), ref.trace_applied)
        np.testing.assert_array_equal(tr[2][:k].cpu().numpy(), ref.trace_objective)


def test_sequential_hand_trace_and_cap_on_gpu():
    with open(GOLDEN) as fh:
        t = {x["name"]: x for x in json.load(fh)["traces"]}["n3_identity_sequential"]
    a = np.array(t["a"], np.int32)
    tr = _trace_tensors(8)
    st, sig, f, stats = B.dgs_solve_ex(_cuda(a), init=B.DGS_INIT_IDENTITY, algorithm=B.DGS_ALG_SEQUENTIAL, trace=tr)
    assert st == B.DGS_OK
    assert sig.cpu().tolist() == t["tau"] and f == t["objective"] and stats["sweeps"] == t["sweeps"]
    assert tr[1][:3].cpu().tolist() == t["applied"]
    big = _make("peer", 300, 4)
    for cap in (1, 5, 40):
        ref = oracle.dgs_sequential(big, max_iters=cap)
        st, sig, f, stats = B.dgs_solve_ex(_cuda(big), max_sweeps=cap, algorithm=B.DGS_ALG_SEQUENTIAL)
        assert st == (B.DGS_TIMEOUT if ref.status == oracle.TIMEOUT else B.DGS_OK)
        np.testing.assert_array_equal(sig.cpu().numpy(), ref.tau)
        assert f == ref.objective and stats["sweeps"] == ref.sweeps
    assert B.dgs_solve_batched([_cuda(big)], algorithm=B.DGS_ALG_SEQUENTIAL)[0] == B.DGS_ERR_INVALID


# ------------------------------- rectangular instances (moves to free jobs)
RECT_CASES = [(1, 5, 0), (3, 7, 1), (64, 100, 2), (100, 64, 3), (130, 257, 4), (300, 129, 5), (257, 257, 6)]


@pytest.mark.parametrize("n,m,seed", RECT_CASES)
def test_rect_matches_oracle(n, m, seed):
    rng = np.random.default_rng(seed)
    a = rng.integers(-50, 1000, size=(n, m), dtype=np.int32)
    for algorithm, init, reeval in ((0, oracle.INIT_GREEDY, oracle.REEVAL_BOX), (0, oracle.INIT_RANDOM, oracle.REEVAL_ALL),
                                    (1, oracle.INIT_GREEDY, oracle.REEVAL_BOX)):
        st_o, assign_o, f_o, sweeps_o = oracle.dgs_rect(a, algorithm=algorithm, init=init, seed=seed, reeval=reeval)
        assert st_o == oracle.OK
        st, assign, f, stats = B.dgs_solve_rect(_cuda(a), algorithm=algorithm, init=init, seed=seed, reeval=reeval)
        assert st == B.DGS_OK, (B.dgs_status_string(st), B.dgs_last_cuda_error())
        np.testing.assert_array_equal(assign.cpu().numpy(), assign_o)
        assert f == f_o and stats["sweeps"] == sweeps_o


def test_rect_rejects_user_start_and_bad_sizes():
    a = _cuda(np.ones((3, 5), np.int32))
    assert B.dgs_solve_rect(a, init=B.DGS_INIT_USER, init_sigma=_cuda(np.arange(5)))[0] == B.DGS_ERR_INVALID
    assert B.dgs_solve_rect(torch.zeros((0, 5), dtype=torch.int32, device="cuda"))[0] == B.DGS_ERR_INVALID
