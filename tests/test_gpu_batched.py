"""Batched and served solves (C ABI: dgs_solve_batched, dgs_server_*) against
the oracle and against the single-instance solve, instance by instance.

Integer work throughout: every instance's assignment, objective, sweep count
and committed exchanges must be bit-identical to the oracle (small sizes) or
to dgs_solve_ex on the instance alone (larger sizes), whatever the mix of
sizes it was solved in.
"""
import os
import subprocess
import sys
import time

import numpy as np
import pytest
import torch

import oracle
from paper_1106_5694_gb300 import binding as B
from paper_1106_5694_gb300 import inputs

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1106_5694_gb300 import build_ext
    build_ext.build()
    oracle.build()
    B.load()


def _make(kind, n, seed):
    if kind == "uniform":
        return inputs.uniform(n, 0, 1000, seed)
    if kind == "ties":
        return inputs.uniform(n, 0, 4, seed)
    if kind == "peer":
        return inputs.peer_shaped(n, seed)
    if kind == "wide":
        return inputs.uniform(n, -(10**8), 10**8, seed)
    raise ValueError(kind)


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


MIXED = [("uniform", 1, 0), ("ties", 2, 1), ("peer", 3, 2), ("uniform", 7, 3), ("wide", 33, 4), ("peer", 64, 5),
         ("ties", 65, 6), ("uniform", 130, 7), ("peer", 257, 8), ("wide", 301, 9), ("uniform", 513, 10),
         ("peer", 640, 11), ("ties", 200, 12), ("uniform", 1000, 13)]


def test_batched_mixed_sizes_equal_oracle():
    mats = [_make(*c) for c in MIXED]
    st, sigs, objs, sts, stats = B.dgs_solve_batched([_cuda(a) for a in mats])
    assert st == B.DGS_OK, (B.dgs_status_string(st), B.dgs_last_cuda_error())
    for a, sig, f, s, stt, case in zip(mats, sigs, objs, sts, stats, MIXED):
        ref = oracle.dgs_parallel(a)
        assert s == B.DGS_OK, case
        np.testing.assert_array_equal(sig.cpu().numpy(), ref.tau, err_msg=str(case))
        assert f == ref.objective, case
        assert stt["sweeps"] == ref.sweeps, case
        assert stt["swaps_applied"] == ref.swaps_applied, case


def test_batched_equals_single_solves_peer_log_uniform():
    ns = inputs.batched_sizes(40, 64, 2048, seed=3)
    mats = [inputs.peer_shaped(int(n), 100 + k) for k, n in enumerate(ns)]
    dev = [_cuda(a) for a in mats]
    st, sigs, objs, sts, stats = B.dgs_solve_batched(dev)
    assert st == B.DGS_OK, B.dgs_last_cuda_error()
    for a_t, sig, f, stt in zip(dev, sigs, objs, stats):
        st1, sig1, f1, s1 = B.dgs_solve_ex(a_t)
        assert st1 == B.DGS_OK
        assert torch.equal(sig, sig1)
        assert f == f1 and stt["sweeps"] == s1["sweeps"] and stt["swaps_applied"] == s1["swaps_applied"]
        assert stt["initial_objective"] == s1["initial_objective"]


def test_batched_identity_start_and_sweep_cap_equal_oracle():
    cases = [("uniform", 150, 4), ("peer", 97, 5), ("ties", 64, 6), ("uniform", 300, 9)]
    mats = [_make(*c) for c in cases]
    st, sigs, objs, sts, _ = B.dgs_solve_batched([_cuda(a) for a in mats], init=B.DGS_INIT_IDENTITY)
    assert st == B.DGS_OK
    for a, sig, f in zip(mats, sigs, objs):
        ref = oracle.dgs_parallel(a, init=oracle.INIT_IDENTITY)
        np.testing.assert_array_equal(sig.cpu().numpy(), ref.tau)
        assert f == ref.objective
    for cap in (1, 3):
        st, sigs, objs, sts, stats = B.dgs_solve_batched([_cuda(a) for a in mats], max_sweeps=cap)
        for a, sig, f, s, stt in zip(mats, sigs, objs, sts, stats):
            ref = oracle.dgs_parallel(a, max_sweeps=cap)
            assert s == (B.DGS_TIMEOUT if ref.status == oracle.TIMEOUT else B.DGS_OK)
            np.testing.assert_array_equal(sig.cpu().numpy(), ref.tau)
            assert f == ref.objective and stt["sweeps"] == ref.sweeps


def test_batched_errors_are_per_instance():
    good = _make("uniform", 40, 0)
    bad = good.copy()
    bad[3, 4] = 1 << 29
    st, sigs, objs, sts, _ = B.dgs_solve_batched([_cuda(good), _cuda(bad), _cuda(good)])
    assert st == B.DGS_ERR_RANGE
    assert sts == [B.DGS_OK, B.DGS_ERR_RANGE, B.DGS_OK]
    ref = oracle.dgs_parallel(good)
    for k in (0, 2):
        np.testing.assert_array_equal(sigs[k].cpu().numpy(), ref.tau)
        assert objs[k] == ref.objective
    # options the batched entry point does not take
    st, *_ = B.dgs_solve_batched([_cuda(good)], init=B.DGS_INIT_USER, init_sigma=_cuda(np.arange(40)))
    assert st == B.DGS_ERR_INVALID
    too_big = torch.zeros((2, 2), dtype=torch.int32, device="cuda")
    assert B.dgs_solve_batched([too_big])[0] == B.DGS_OK


def test_batched_unaligned_and_ragged_inputs():
    # a matrix whose rows are not 16-byte aligned (n % 4 != 0) and one at an
    # odd offset inside a larger buffer: both are re-pitched on the device
    a = _make("peer", 203, 21)
    base = torch.zeros(203 * 203 + 1, dtype=torch.int32, device="cuda")
    base[1:] = torch.from_numpy(a.reshape(-1)).cuda()
    shifted = base[1:].view(203, 203)
    b = _make("uniform", 256, 22)
    st, sigs, objs, sts, _ = B.dgs_solve_batched([shifted, _cuda(b), _cuda(a)])
    assert st == B.DGS_OK
    for m, sig, f in zip((a, b, a), sigs, objs):
        ref = oracle.dgs_parallel(m)
        np.testing.assert_array_equal(sig.cpu().numpy(), ref.tau)
        assert f == ref.objective


_KNOB_SCRIPT = r"""
import sys, json, numpy as np, torch
sys.path.insert(0, {root!r})
from paper_1106_5694_gb300 import binding as B, inputs
mats = []
for kind, n, seed in {cases!r}:
    mats.append(inputs.peer_shaped(n, seed) if kind == "peer" else inputs.uniform(n, 0, 1000, seed))
st, sigs, objs, sts, stats = B.dgs_solve_batched([torch.from_numpy(a).cuda() for a in mats])
print(json.dumps([st, objs, [s["sweeps"] for s in stats], [g.cpu().tolist() for g in sigs]]))
"""


@pytest.mark.parametrize("env", [{"DGS_UPDATE_POLICY": "1"}, {"DGS_UPDATE_POLICY": "2"}, {"DGS_CTL_MODE": "0"},
                                 {"DGS_SHORT_WRAPS": "1"}, {"DGS_EXACT_KEYS": "1"}, {"DGS_CTL_COMPACT_MIN": "1"}])
def test_batched_internal_paths_agree_with_oracle(env):
    import json
    cases = [("uniform", 300, 1), ("peer", 257, 2), ("uniform", 513, 3), ("peer", 64, 4)]
    r = subprocess.run([sys.executable, "-c", _KNOB_SCRIPT.format(root=ROOT, cases=cases)],
                       env=dict(os.environ, **env), capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    st, objs, sweeps, taus = json.loads(r.stdout.strip().splitlines()[-1])
    assert st == B.DGS_OK
    for (kind, n, seed), f, sw, tau in zip(cases, objs, sweeps, taus):
        a = inputs.peer_shaped(n, seed) if kind == "peer" else inputs.uniform(n, 0, 1000, seed)
        ref = oracle.dgs_parallel(a)
        assert f == ref.objective and sw == ref.sweeps and tau == ref.tau.tolist()


# -------------------------------------------------------------------- server
def _alone(a_np):
    st, sig, f = B.dgs_solve(_cuda(a_np))
    assert st == B.DGS_OK
    return sig.cpu().numpy(), f


def test_server_results_equal_alone_in_a_staggered_mix():
    ns = [300, 64, 1024, 7, 513, 2048, 130, 900]
    mats = [inputs.peer_shaped(n, 200 + k) if k % 2 == 0 else inputs.uniform(n, 0, 1000, 200 + k)
            for k, n in enumerate(ns)]
    want = [_alone(a) for a in mats]
    with B.Server(budget_bytes=8 << 30) as srv:
        tickets = []
        for k, a in enumerate(mats):
            # host and device inputs, arriving while earlier requests run
            st, t = srv.dgs_submit(a if k % 3 else _cuda(a))
            assert st == B.DGS_OK
            tickets.append(t)
            time.sleep(0.002 * (k % 3))
        for t, (sig_w, f_w) in zip(tickets, want):
            st, sig, f, stats, times = srv.dgs_server_wait(t, timeout_us=120_000_000)
            assert st == B.DGS_OK, B.dgs_status_string(st)
            np.testing.assert_array_equal(sig, sig_w)
            assert f == f_w
            order = [times[k] for k in ("submit_ns", "admit_ns", "upload_ns", "ready_ns", "start_ns", "done_ns")]
            assert order == sorted(order) and order[0] > 0
        st, info = srv.dgs_server_get_info()
        assert st == B.DGS_OK and info["completed"] == len(mats) and info["resident"] == 0
        assert info["bytes_in_use"] == 0 and info["steps"] > 0


def test_server_budget_admits_one_at_a_time_and_rejects_oversize():
    mats = [inputs.peer_shaped(n, 300 + n) for n in (400, 500, 600)]
    want = [_alone(a) for a in mats]
    budget = max(B.dgs_server_request_bytes(a.shape[0]) for a in mats)
    with B.Server(budget_bytes=budget) as srv:
        big = np.zeros((1000, 1000), np.int32)
        assert srv.dgs_submit(big)[0] == B.DGS_ERR_BUSY
        tickets = [srv.dgs_submit(a)[1] for a in mats]
        peak_resident = 0
        pending = set(tickets)
        results = {}
        t0 = time.time()
        while pending and time.time() - t0 < 120:
            peak_resident = max(peak_resident, srv.dgs_server_get_info()[1]["resident"])
            for t in list(pending):
                st, sig, f, _, _ = srv.dgs_poll(t)
                if st != B.DGS_PENDING:
                    results[t] = (st, sig, f)
                    pending.discard(t)
            time.sleep(0.0005)
        assert not pending
        assert peak_resident <= 1
        for t, (sig_w, f_w) in zip(tickets, want):
            st, sig, f = results[t]
            assert st == B.DGS_OK
            np.testing.assert_array_equal(sig, sig_w)
            assert f == f_w
        assert srv.dgs_poll(tickets[0])[0] == B.DGS_ERR_INVALID  # taken already


def test_server_range_error_and_continued_service():
    a = inputs.uniform(50, 0, 1000, 1)
    bad = a.copy()
    bad[0, 0] = -(1 << 29)
    with B.Server(budget_bytes=1 << 30) as srv:
        t_bad = srv.dgs_submit(bad)[1]
        t_ok = srv.dgs_submit(a)[1]
        assert srv.dgs_server_wait(t_bad)[0] == B.DGS_ERR_RANGE
        st, sig, f, _, _ = srv.dgs_server_wait(t_ok)
        assert st == B.DGS_OK
        ref = oracle.dgs_parallel(a)
        np.testing.assert_array_equal(sig, ref.tau)
        assert f == ref.objective


def test_server_warm_start_and_per_request_options():
    """A periodic re-solve: the previous assignment of a slowly changing
    matrix is the start of the next solve (dgs_submit_ex); results equal the
    single solve with the same options."""
    base = inputs.peer_shaped(500, 41)
    st, sig0, _ = B.dgs_solve(_cuda(base))
    prev = sig0.cpu().numpy()
    rng = np.random.default_rng(5)
    moved = base + rng.integers(0, 200, size=base.shape, dtype=np.int32)  # the peers' benefits drift
    cases = [dict(init_sigma=prev), dict(init=B.DGS_INIT_RANDOM, seed=9, reeval=B.DGS_REEVAL_ALL),
             dict(init=B.DGS_INIT_IDENTITY, max_sweeps=3)]
    with B.Server(budget_bytes=2 << 30) as srv:
        tickets = []
        for k, c in enumerate(cases):
            if k == 0:  # device memory for the first: matrix and start
                t = srv.dgs_submit_ex(_cuda(moved), init_sigma=_cuda(prev))
            else:
                t = srv.dgs_submit_ex(moved, **c)
            assert t[0] == B.DGS_OK
            tickets.append(t[1])
        bad = prev.copy()
        bad[0] = bad[1]
        t_bad = srv.dgs_submit_ex(moved, init_sigma=bad)[1]
        for t, c in zip(tickets, cases):
            st, sig, f, stats, _ = srv.dgs_server_wait(t)
            single = dict(c)
            if "init_sigma" in single:
                single["init_sigma"] = _cuda(single["init_sigma"])
                single["init"] = B.DGS_INIT_USER
            st1, sig1, f1, stats1 = B.dgs_solve_ex(_cuda(moved), **single)
            assert st == st1
            np.testing.assert_array_equal(sig, sig1.cpu().numpy())
            assert f == f1 and stats["sweeps"] == stats1["sweeps"]
        assert srv.dgs_server_wait(t_bad)[0] == B.DGS_ERR_INVALID
        assert srv.dgs_submit_ex(moved, algorithm=B.DGS_ALG_SEQUENTIAL)[0] == B.DGS_ERR_INVALID
