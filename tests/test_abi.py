"""The C-ABI library builds, loads and exports every entry point of include/pngf.h (CPU).

Only host-side logic runs here: argument checks and the workspace query need
no GPU; no compute entry point is called.
"""
import ctypes
import os
import re

import pytest

from paper_2501_18054_gb300 import build as B
from paper_2501_18054_gb300 import pngf as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    return B.build()


def _declared():
    text = open(os.path.join(ROOT, "include", "pngf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pngf_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(built):
    lib = ctypes.CDLL(built["libpngf.so"])
    declared = _declared()
    assert len(declared) >= 14
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing
    assert set(P.exported_symbols()) <= set(declared)


def test_peaks_library_exports(built):
    lib = ctypes.CDLL(built["libpngf_peaks.so"])
    assert hasattr(lib, "pngf_peak_fp64_gflops") and hasattr(lib, "pngf_peak_fp32_gflops")


def test_workspace_query_and_argument_checks(built):
    cfg = P.make_config(4096, 2)
    ws = P.pngf_workspace_size(cfg)
    n = 4096
    # at least W, the LU factors and a snapshot of W in complex128
    assert ws >= 3 * n * n * 16
    small = P.pngf_workspace_size(P.make_config(100, 2))
    assert 0 < small < ws
    for bad in (dict(n_d=0), dict(n_d=40000), dict(n_o=0), dict(n_o=9)):
        c = P.make_config(bad.get("n_d", 64), bad.get("n_o", 2))
        with pytest.raises(P.PngfError) as ei:
            P.pngf_workspace_size(c)
        assert ei.value.status == P.PNGF_EINVAL
    c = P.make_config(64, 2)
    c.precision = 7
    with pytest.raises(P.PngfError):
        P.pngf_workspace_size(c)
    c = P.make_config(64, 2)
    c.tau = -1.0
    with pytest.raises(P.PngfError):
        P.pngf_workspace_size(c)


def test_null_handles_are_rejected(built):
    L = P.lib()
    assert L.pngf_factor(None, None) == P.PNGF_EINVAL
    assert L.pngf_accept_flip(None, 0) == P.PNGF_EINVAL
    assert L.pngf_dbs_sweep(None, 1, None, None, None, 0, None) == P.PNGF_EINVAL
    assert L.pngf_eval_ports(None, None, None) == P.PNGF_EINVAL
    assert L.pngf_sync(None) == P.PNGF_EINVAL
    out = ctypes.c_void_p()
    assert L.pngf_create(None, None, None, None, None, None, None, 0, None, ctypes.byref(out)) == P.PNGF_EINVAL


def test_status_strings(built):
    for s in range(9):
        assert P.pngf_status_string(s) and P.pngf_status_string(s) != "unknown status"
    assert P.pngf_status_string(99) == "unknown status"
