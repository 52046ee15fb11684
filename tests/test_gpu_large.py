"""Sizes beyond the oracle's reach (n = 40000, and the maximum 2^17): the
greedy start by deferred acceptance and a full solve there, checked by
properties that hold at any size.

The global greedy assignment (reading R1) is characterised without running
it: under the strict order of pairs (benefit desc, agent asc, job asc), a
perfect matching is the greedy one exactly when every pair outside it is
preceded by the matched pair of its agent or of its job.  (The first pair of
the order must be matched, and inductively each next greedy pair, if it were
not matched, would be preceded by a matched pair sharing a vertex that the
greedy process had already used.)  The checker is itself checked against the
oracle's greedy start and against a planted swap."""
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
    oracle.build()
    B.load()


def _keys(vals, rows, cols):
    """Order key of pairs: larger = earlier (benefit desc, agent asc, job asc)."""
    return (vals.long() << 34) | ((131071 - rows.long()) << 17) | (131071 - cols.long())


def is_global_greedy(a, tau, block=1024):
    n = a.shape[0]
    dev = a.device
    t = tau.long()
    sigma = torch.empty_like(t)
    sigma[t] = torch.arange(n, device=dev)
    ar = torch.arange(n, device=dev)
    rowkey = _keys(a[ar, t], ar, t)          # the matched pair of each agent
    colkey = _keys(a[sigma, ar], sigma, ar)  # the matched pair of each job
    for r0 in range(0, n, block):
        r1 = min(n, r0 + block)
        rows = ar[r0:r1, None]
        k = _keys(a[r0:r1], rows.expand(-1, n), ar[None, :].expand(r1 - r0, -1))
        bound = torch.maximum(rowkey[r0:r1, None], colkey[None, :])
        matched = ar[None, :] == t[r0:r1, None]
        if not bool(torch.all(k <= bound)) or not bool(torch.all((k == bound) == matched)):
            return False
    return True


def test_greedy_characterisation_against_the_oracle_and_a_planted_swap():
    a_np = inputs.uniform(3000, 0, 50, 3)  # heavy ties
    a = torch.from_numpy(a_np).cuda()
    tau = torch.from_numpy(oracle.greedy_init(a_np)).cuda()
    assert is_global_greedy(a, tau)
    wrong = tau.clone()
    wrong[[10, 20]] = wrong[[20, 10]]
    assert not is_global_greedy(a, wrong)


@pytest.mark.parametrize("n,hi", [(40000, 1000), (40003, 10**6)])
def test_greedy_start_at_large_n_is_the_global_greedy(n, hi):
    g = torch.Generator(device="cuda")
    g.manual_seed(n)
    a = torch.randint(0, hi, (n, n), dtype=torch.int32, device="cuda", generator=g)
    st, tau = B.dgs_greedy_init(a)
    assert st == B.DGS_OK, B.dgs_status_string(st)
    assert torch.equal(torch.sort(tau.long()).values, torch.arange(n, device="cuda"))
    assert is_global_greedy(a, tau)
    del a
    torch.cuda.empty_cache()


def test_solve_at_n_40000():
    n = 40000
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    a = torch.randint(0, 10**6, (n, n), dtype=torch.int32, device="cuda", generator=g)
    st, sig, f, stats = B.dgs_solve_ex(a)
    assert st == B.DGS_OK, B.dgs_status_string(st)
    s64 = sig.long()
    assert torch.equal(torch.sort(s64).values, torch.arange(n, device="cuda"))
    d = a[torch.arange(n, device="cuda"), s64].long()
    assert f == int(d.sum().item()) and f >= stats["initial_objective"]
    best = -1
    for r0 in range(0, n, 1024):  # no improving 2-exchange
        cross = a[r0:r0 + 1024][:, s64].long()
        back = a[:, s64[r0:r0 + 1024]].long().T
        best = max(best, int((cross + back - d[r0:r0 + 1024, None] - d[None, :]).max().item()))
    assert best <= 0
    del a
    torch.cuda.empty_cache()


def test_solve_at_the_maximum_size():
    """n = 2^17 (the largest n the library accepts; 68.7 GB per matrix): a
    planted optimum (benefit 2000 on a seeded permutation, others below 100)
    is found exactly, and nothing improves it."""
    n = 1 << 17
    g = torch.Generator(device="cuda")
    g.manual_seed(17)
    a = torch.randint(0, 100, (n, n), dtype=torch.int32, device="cuda", generator=g)
    perm = torch.randperm(n, device="cuda", generator=g)
    ar = torch.arange(n, device="cuda")
    a[ar, perm] = 2000
    st, sig, f, stats = B.dgs_solve_ex(a)
    assert st == B.DGS_OK, B.dgs_status_string(st) + " " + B.dgs_last_cuda_error()
    assert torch.equal(sig.long(), perm) and f == 2000 * n
    assert stats["sweeps"] == 0 and stats["greedy_rounds"] == 1
    s64 = sig.long()
    best = -1
    for r0 in range(0, n, 1024):  # no improving 2-exchange
        cross = a[r0:r0 + 1024][:, s64].long()
        back = a[:, s64[r0:r0 + 1024]].long().T
        best = max(best, int((cross + back - 2000 - 2000).max().item()))
    assert best <= 0
    del a, cross, back
    torch.cuda.empty_cache()
    assert B.dgs_release_cached_memory() == B.DGS_OK
