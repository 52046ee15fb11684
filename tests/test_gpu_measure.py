"""dgs_read_bandwidth: the read-rate probe behind the L2 roofline."""
import pytest
import torch

from paper_1106_5694_gb300 import binding as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1106_5694_gb300 import build_ext
    build_ext.build()
    B.load()


def test_read_bandwidth_l2_and_hbm_sized_buffers():
    small = torch.ones(16 << 20, dtype=torch.int32, device="cuda")   # 64 MiB: fits in L2
    large = torch.ones(256 << 20, dtype=torch.int32, device="cuda")  # 1 GiB: does not
    st_s, l2 = B.dgs_read_bandwidth(small, repeats=20)
    st_l, hbm = B.dgs_read_bandwidth(large, repeats=5)
    assert st_s == B.DGS_OK and st_l == B.DGS_OK
    # positive, finite, and the L2-resident buffer reads faster than one that
    # streams from HBM
    assert 0 < hbm < l2 < 1e6
    assert torch.all(small == 1) and torch.all(large[:1024] == 1)  # nothing written


def test_read_bandwidth_rejects_bad_arguments():
    lib = B.load()
    import ctypes
    x = torch.zeros(1024, dtype=torch.int32, device="cuda")
    out = ctypes.c_double(0.0)
    p = ctypes.c_void_p(x.data_ptr())
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.dgs_read_bandwidth(None, 4096, 1, ctypes.byref(out), s) == B.DGS_ERR_INVALID
    assert lib.dgs_read_bandwidth(p, 4095, 1, ctypes.byref(out), s) == B.DGS_ERR_INVALID
    assert lib.dgs_read_bandwidth(p, 0, 1, ctypes.byref(out), s) == B.DGS_ERR_INVALID
    assert lib.dgs_read_bandwidth(p, 4096, 0, ctypes.byref(out), s) == B.DGS_ERR_INVALID
    assert lib.dgs_read_bandwidth(ctypes.c_void_p(x.data_ptr() + 4), 4096, 1, ctypes.byref(out), s) == \
        B.DGS_ERR_INVALID
    assert lib.dgs_read_bandwidth(p, 4096, 1, None, s) == B.DGS_ERR_INVALID


def test_release_cached_memory_after_solves():
    """Solves reuse the library pool's cached workspace; releasing it keeps
    later solves correct."""
    from paper_1106_5694_gb300 import inputs
    a = torch.from_numpy(inputs.peer_shaped(700, 3)).cuda()
    st1, sig1, f1, _ = B.dgs_solve_ex(a)
    st2, sig2, f2, _ = B.dgs_solve_ex(a)
    free_before = torch.cuda.mem_get_info()[0]
    assert B.dgs_release_cached_memory() == B.DGS_OK
    free_after = torch.cuda.mem_get_info()[0]
    st3, sig3, f3, _ = B.dgs_solve_ex(a)
    assert st1 == st2 == st3 == B.DGS_OK and f1 == f2 == f3
    assert torch.equal(sig1, sig2) and torch.equal(sig1, sig3)
    assert free_after >= free_before
