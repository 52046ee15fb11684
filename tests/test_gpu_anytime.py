"""Anytime behaviour and failure paths of the solver, with no GPU fault.

Section 3 of the paper notes that DGS can be stopped at any point and still
hold a valid assignment; here that is the deadline option: a solve whose
deadline passes returns DGS_TIMEOUT with the assignment reached so far, its
exact objective, and that assignment is the oracle's after the same number of
sweeps.  An allocation failure (a fake of the failing allocation, made on the
host) returns DGS_ERR_OOM and leaves the library usable; a queued server
request can be withdrawn, and one that can never fit the budget is refused.
"""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1106_5694_gb300 import binding as B
from paper_1106_5694_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1106_5694_gb300 import build_ext
    build_ext.build()
    B.load()


def _objective(a, sig):
    return int(a[np.arange(a.shape[0]), sig].astype(np.int64).sum())


def test_deadline_passed_before_the_first_sweep_returns_the_start():
    a = inputs.uniform(3000, 0, 10**6, seed=21)
    at = torch.from_numpy(a).cuda()
    st, sig, f, stats = B.dgs_solve_ex(at, deadline_us=1)
    assert st == B.DGS_TIMEOUT and stats["status"] == B.DGS_TIMEOUT
    assert stats["sweeps"] == 0
    s = sig.cpu().numpy()
    assert np.array_equal(np.sort(s), np.arange(3000)) and f == _objective(a, s)
    st_g, g = B.dgs_greedy_init(at)
    assert st_g == B.DGS_OK and np.array_equal(s, g.cpu().numpy())
    assert f == stats["initial_objective"]


def test_deadline_mid_solve_returns_the_oracle_prefix():
    a = inputs.uniform(900, 0, 10**6, seed=22)
    at = torch.from_numpy(a).cuda()
    st, _, _, full = B.dgs_solve_ex(at, profile=1)
    assert st == B.DGS_OK and full["sweeps"] > 20
    for frac in (0.3, 0.6):
        deadline = max(1, int(full["solve_ms"] * 1e3 * frac))
        st, sig, f, stats = B.dgs_solve_ex(at, deadline_us=deadline)
        s = sig.cpu().numpy()
        assert np.array_equal(np.sort(s), np.arange(900)) and f == _objective(a, s)
        if st == B.DGS_OK:  # finished before the deadline
            ref = oracle.dgs_parallel(a)
        else:
            assert st == B.DGS_TIMEOUT
            assert f >= stats["initial_objective"]
            if stats["sweeps"] == 0:
                ref_tau = oracle.greedy_init(a)
                assert np.array_equal(s, ref_tau)
                continue
            ref = oracle.dgs_parallel(a, max_sweeps=stats["sweeps"])
        np.testing.assert_array_equal(s, ref.tau)
        assert f == ref.objective and stats["sweeps"] == ref.sweeps


def test_allocation_failure_is_reported_and_the_library_stays_usable(monkeypatch):
    a = inputs.peer_shaped(512, seed=23)
    at = torch.from_numpy(a).cuda()
    monkeypatch.setenv("DGS_FAKE_OOM_BYTES", str(1 << 20))  # every solve workspace of n = 512 is larger
    st, *_ = B.dgs_solve_ex(at)
    assert st == B.DGS_ERR_OOM
    assert "workspace" in B.dgs_last_cuda_error()
    st, *_ = B.dgs_solve_rect(at[:, :400].contiguous())
    assert st == B.DGS_ERR_OOM
    monkeypatch.delenv("DGS_FAKE_OOM_BYTES")
    st, sig, f, _ = B.dgs_solve_ex(at)
    ref = oracle.dgs_parallel(a)
    assert st == B.DGS_OK and f == ref.objective
    np.testing.assert_array_equal(sig.cpu().numpy(), ref.tau)


def test_server_cancels_a_queued_request_and_refuses_one_that_never_fits():
    # uniform n = 4096 instances take over a thousand sweeps each, so while
    # the first one runs the others wait for the budget (room for one)
    n = 4096
    budget = B.dgs_server_request_bytes(n) + B.dgs_server_request_bytes(n) // 2
    mats = [torch.from_numpy(inputs.uniform(n, 0, 10**6, seed=30 + k)).cuda() for k in range(3)]
    with B.dgs_server_create(budget) as srv:
        big = torch.zeros((6000, 6000), dtype=torch.int32, device="cuda")
        assert srv.dgs_submit(big)[0] == B.DGS_ERR_BUSY
        tickets = []
        for m in mats:
            st, t = srv.dgs_submit(m)
            assert st == B.DGS_OK
            tickets.append(t)
        assert srv.dgs_cancel(tickets[2]) == B.DGS_OK
        assert srv.dgs_server_wait(tickets[2])[0] == B.DGS_CANCELLED
        assert srv.dgs_cancel(tickets[2]) == B.DGS_ERR_INVALID  # forgotten after the wait
        assert srv.dgs_cancel(987654321) == B.DGS_ERR_INVALID
        for t, m in zip(tickets[:2], mats[:2]):
            st, sig, f, *_ = srv.dgs_server_wait(t)
            st1, sig1, f1, _ = B.dgs_solve_ex(m)
            assert st == st1 == B.DGS_OK and f == f1
            np.testing.assert_array_equal(np.asarray(sig), sig1.cpu().numpy())
