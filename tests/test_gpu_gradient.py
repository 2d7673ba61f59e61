"""The objective gradient (pngf_gradient) against the CPU oracle.

The oracle's objective_gradient is pinned to central differences of the
reduced-system evaluation and to the one-pixel closed form (CPU tests).  Bars:
FP64 contexts 1e-10 relative to the largest entry (1e-9 on the lossy-metal
case, cond(M) ~ 5e6); a mixed context right after its FP64 factor the same,
and after a mixed search 1e-4 (its state between refreshes carries FP32-level
error, the same bar as its S-parameters).
"""
import numpy as np
import pytest

from paper_2501_18054_gb300 import workloads as W
import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2501_18054_gb300 import build as B
    B.build()
    from paper_2501_18054_gb300 import pngf
    return pngf


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("name,kind,seed", [("fdfd64", 0, 3), ("fdfd64", 1, 4), ("fdfd128_metal", 0, 5),
                                             ("fdfd128_metal", 1, 6)])
def test_gradient_parity_fp64(P, name, kind, seed):
    case = W.get_case(name)
    case.obj_kind = kind
    b = W.random_design(case.n_d, seed)
    ctx = P.DbsContext(case)
    ctx.factor(b)
    g, dod = ctx.gradient(want_dodrho=True)
    p = O.Problem.from_case(case)
    want = O.objective_gradient(p, b.astype(np.float64))
    tol = 1e-9 if name == "fdfd128_metal" else 1e-10
    assert rel(g, want) < tol
    v = case.dv * b
    T = O.port_projection(case.G_dd, case.G_od, v)
    e = O.evaluate(p, b).e
    assert rel(dod, T * (e * case.dv)[None, :]) < tol
    ctx.close()


def test_gradient_after_search_and_on_mixed(P):
    case = W.get_case("fdfd64")
    b0 = W.random_design(case.n_d, 0)
    for prec, tol_after in ((P.PNGF_FP64, 1e-9), (P.PNGF_MIXED, 1e-4)):
        kw = dict(precision=prec, refresh_k=16)
        if prec == P.PNGF_MIXED:
            kw.update(delay_r=8, tensor_fold=1)
        ctx = P.DbsContext(case, **kw)
        ctx.factor(b0)
        p = O.Problem.from_case(case)
        assert rel(ctx.gradient(), O.objective_gradient(p, b0.astype(np.float64))) < 1e-10
        ctx.dbs_sweep(1)
        b = ctx.design()
        assert rel(ctx.gradient(), O.objective_gradient(p, b.astype(np.float64))) < tol_after
        ctx.close()
