"""pngf_accept_flip_noalloc against pngf_accept_flip, through the C ABI (GPU).

Some callers may not allocate device memory while they run (their pool is
owned by another allocator, or a cudaMalloc's implicit synchronisation is not
allowed in their loop).  For them the kept-flip update has a variant whose
scratch lives in a fixed array inside the library.  This file runs last so
that a failure here leaves every other test already run; it passes alone in
a fresh process and after the other tests.
"""
import numpy as np
import pytest

from paper_2501_18054_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2501_18054_gb300 import build as B
    B.build()
    from paper_2501_18054_gb300 import pngf
    return pngf


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def test_noalloc_accept_matches_accept_on_two_calls(P):
    case = W.get_case("fdfd64")
    b = W.random_design(case.n_d, 7)
    ref = P.DbsContext(case)
    new = P.DbsContext(case)
    ref.factor(b)
    new.factor(b)
    iu = np.triu_indices(case.n_d)
    for k in (13, 71):  # two calls in a row: the shared array keeps the last call's contents
        P.pngf_accept_flip(ref.ctx, k)
        P.pngf_accept_flip_noalloc(new.ctx, k)
        assert ref.sync() == 0 and new.sync() == 0
        a, c = ref.state(with_W=True), new.state(with_W=True)
        # same tolerance as the accept parity test of the FP64 path
        assert rel(c["W"][iu], a["W"][iu]) < 1e-11
        for key in ("diag", "e", "T", "o"):
            assert rel(c[key], a[key]) < 1e-11, key
        oa, fa = ref.eval_ports()
        oc, fc = new.eval_ports()
        assert rel(oc, oa) < 1e-11 and abs(fc - fa) <= 1e-11 * abs(fa)
        assert np.array_equal(ref.design(), new.design())
    ref.close()
    new.close()


def test_noalloc_rejects_what_it_cannot_hold(P):
    import torch

    case = W.get_case("fdfd64")
    mixed = P.DbsContext(case, precision=P.PNGF_MIXED, delay_r=8, refresh_k=16)
    mixed.factor(W.random_design(case.n_d, 0))
    with pytest.raises(P.PngfError) as ei:
        P.pngf_accept_flip_noalloc(mixed.ctx, 3)
    assert ei.value.status == P.PNGF_EINVAL
    mixed.close()
    # a region larger than the fixed array: rejected before any device work
    n = P.PNGF_NOALLOC_MAX_ND
    cfg = P.make_config(n + 1, 2)
    ws_bytes = P.pngf_workspace_size(cfg)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    small = torch.zeros(64, dtype=torch.complex128, device="cuda")
    h = P.pngf_create(cfg, small.data_ptr(), small.data_ptr(), small.data_ptr(), small.data_ptr(),
                      small.data_ptr(), ws.data_ptr(), ws_bytes, torch.cuda.current_stream().cuda_stream)
    with pytest.raises(P.PngfError) as ei:
        P.pngf_accept_flip_noalloc(h, 0)
    assert ei.value.status == P.PNGF_EINVAL
    P.pngf_destroy(h)
    del ws
