"""Autotuned launch shapes (C ABI: dgs_autotune, dgs_get_tuning): the tuner
picks a valid shape for the size class, later solves use it, and no shape
changes any result (assignment, objective, sweeps equal to the oracle)."""
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


@pytest.mark.parametrize("n", [300, 1000])
def test_autotune_picks_a_shape_and_solves_stay_exact(n):
    st, r = B.dgs_autotune(n)
    assert st == B.DGS_OK, B.dgs_last_cuda_error()
    assert r["rows_per_thread"] in (4, 8, 16) and r["strip"] >= 0
    assert r["n_lo"] <= n <= r["n_hi"]
    assert len(r["candidates"]) >= 6 and all(c["ms"] > 0 for c in r["candidates"])
    assert r["best_ms"] == min(c["ms"] for c in r["candidates"])
    st, rows, strip, tma = B.dgs_get_tuning(n)
    assert st == B.DGS_OK and (rows, strip, tma) == (r["rows_per_thread"], r["strip"], r["tma"])
    assert {c["tma"] for c in r["candidates"]} == {0, 1}
    for kind, seed in (("peer", 1), ("uniform", 2)):
        a = inputs.peer_shaped(n, seed) if kind == "peer" else inputs.uniform(n, 0, 1000, seed)
        ref = oracle.dgs_parallel(a)
        st, sig, f, stats = B.dgs_solve_ex(torch.from_numpy(a).cuda())
        assert st == B.DGS_OK
        np.testing.assert_array_equal(sig.cpu().numpy(), ref.tau)
        assert f == ref.objective and stats["sweeps"] == ref.sweeps


def test_autotune_rejects_bad_sizes():
    assert B.dgs_autotune(1)[0] == B.DGS_ERR_INVALID
    assert B.dgs_autotune(0)[0] == B.DGS_ERR_INVALID
