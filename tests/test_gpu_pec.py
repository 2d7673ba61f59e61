"""The perfect-conductor (PEC) path (precision PNGF_PEC) against the CPU
oracle's evaluate_pec (the paper's Eq. 2 solved from scratch, pinned to a
full FDFD solve with the metal nodes held at zero field).

Bars as the FP64 path: state and candidate objectives within 1e-10 (1e-9 on
the 1024-pixel region), the accepted-flip sequence equal to the oracle's
while its decision margins exceed 1e-9 |f|.
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


def _block(side_big, x0, side):
    return np.array([(x0 + i) * side_big + (x0 + j) for i in range(side) for j in range(side)])


def _case(name):
    if name == "metal_sub256":
        return W.get_case("fdfd128_metal").sub_case(_block(32, 8, 16), "metal_sub256")
    return W.get_case(name)


def _pec_reference(case, b):
    """H, W = G - G H G, total field and ports of design b, from direct solves."""
    n = case.n_d
    M = np.flatnonzero(b)
    H = np.zeros((n, n), complex)
    if len(M):
        H[np.ix_(M, M)] = np.linalg.inv(case.G_dd[np.ix_(M, M)])
    Wp = case.G_dd - case.G_dd @ H @ case.G_dd
    T = case.G_od - case.G_od @ H @ case.G_dd
    return Wp, T


@pytest.mark.parametrize("name,seed", [("fdfd64", 1), ("metal_sub256", 2), ("fdfd128_metal", 3)])
def test_pec_factor_state_parity(P, name, seed):
    case = _case(name)
    b = W.random_design(case.n_d, seed)
    tol = 1e-9 if case.n_d > 256 else 1e-10
    ctx = P.DbsContext(case, precision=P.PNGF_PEC)
    ctx.factor(b)
    st = ctx.state(with_W=True)
    ev = O.evaluate_pec(O.Problem.from_case(case), b)
    Wp, T = _pec_reference(case, b)
    iu = np.triu_indices(case.n_d)
    assert rel(st["W"][iu], Wp[iu]) < tol
    assert rel(st["diag"], np.diag(Wp)) < tol
    assert rel(st["e"], ev.e) < tol
    assert rel(st["T"], T) < tol
    o, f = ctx.eval_ports()
    assert rel(o, ev.o) < tol
    assert abs(f - ev.f) <= tol * abs(ev.f)
    assert np.array_equal(ctx.design(), b)
    ctx.close()


@pytest.mark.parametrize("name", ["fdfd64", "fdfd128_metal"])
def test_pec_score_flips_parity(P, name):
    case = _case(name)
    b = W.random_design(case.n_d, 5)
    ctx = P.DbsContext(case, precision=P.PNGF_PEC)
    ctx.factor(b)
    px = np.arange(case.n_d) if case.n_d <= 256 else np.arange(0, case.n_d, 7)
    f = ctx.score_flips(px)
    ref = O.candidate_objectives(O.Problem.from_case(case), b, px, O.evaluate_pec)
    tol = 5e-9 if case.n_d > 256 else 1e-9
    assert np.max(np.abs(f - ref) / np.abs(ref)) < tol
    ctx.close()


def test_pec_accept_both_directions(P):
    case = _case("metal_sub256")
    b = W.random_design(case.n_d, 6)
    ctx = P.DbsContext(case, precision=P.PNGF_PEC)
    ctx.factor(b)
    on, off = int(np.flatnonzero(b)[3]), int(np.flatnonzero(b == 0)[5])
    for k in (on, off, on):
        ctx.accept_flip(k)
        b[k] ^= 1
        st = ctx.state(with_W=True)
        Wp, T = _pec_reference(case, b)
        iu = np.triu_indices(case.n_d)
        assert rel(st["W"][iu], Wp[iu]) < 1e-10
        assert rel(st["T"], T) < 1e-10
        assert rel(ctx.eval_ports()[0], O.evaluate_pec(O.Problem.from_case(case), b).o) < 1e-10
        assert np.array_equal(ctx.design(), b)
    ctx.close()


PEC_RUNS = {
    "fdfd64_first_raster": ("fdfd64", 0, "raster", O.FIRST_IMPROVEMENT, 6),
    "fdfd64_first_shuffled": ("fdfd64", 1, "shuffled", O.FIRST_IMPROVEMENT, 6),
    "fdfd64_best": ("fdfd64", 2, "raster", O.BEST_IMPROVEMENT, 60),
    "metal_sub256_first_raster": ("metal_sub256", 3, "raster", O.FIRST_IMPROVEMENT, 4),
}


@pytest.mark.parametrize("run", sorted(PEC_RUNS))
def test_pec_dbs_matches_oracle(P, run):
    name, seed, order_kind, mode, sweeps = PEC_RUNS[run]
    case = _case(name)
    n = case.n_d
    order = W.raster_order(n, sweeps) if order_kind == "raster" else W.shuffled_order(n, sweeps, seed=seed)
    b0 = W.random_design(n, seed)
    # tau = 1e-6: in a PEC design some pixels are shielded by the metal around
    # them, and their flips change the objective only at rounding level; the
    # larger threshold rejects them clearly instead of at a near-tie
    ref = O.dbs(O.Problem.from_case(case), b0, order, tau=1e-6, mode=mode, evaluator=O.evaluate_pec)
    assert ref.min_abs_margin > 1e-9 * abs(ref.f)
    pm = P.PNGF_FIRST_IMPROVEMENT if mode == O.FIRST_IMPROVEMENT else P.PNGF_BEST_IMPROVEMENT
    ctx = P.DbsContext(case, precision=P.PNGF_PEC, mode=pm, tau=1e-6)
    ctx.factor(b0)
    ctx.snapshot()
    res = ctx.dbs_sweep(sweeps, order=order if order_kind == "shuffled" else None)
    assert [tuple(int(x) for x in r[:3]) for r in res["trace"]] == [a[:3] for a in ref.accepted]
    f_ref = np.array([a[3] for a in ref.accepted])
    assert np.max(np.abs(res["trace_f"] - f_ref)) <= 1e-9 * np.max(np.abs(f_ref))
    assert np.array_equal(ctx.design(), ref.b)
    assert rel(ctx.eval_ports()[0], ref.o) < 1e-9
    assert res["counters"][1] == ref.n_evals
    # a restored snapshot replays bit for bit
    ctx.restore()
    res2 = ctx.dbs_sweep(sweeps, order=order if order_kind == "shuffled" else None)
    assert np.array_equal(res["trace"], res2["trace"]) and np.array_equal(res["trace_f"], res2["trace_f"])
    ctx.close()


def test_pec_unavailable_calls(P):
    case = _case("fdfd64")
    ctx = P.DbsContext(case, precision=P.PNGF_PEC)
    ctx.factor(W.random_design(case.n_d, 0))
    with pytest.raises(P.PngfError):
        ctx.gradient()
    with pytest.raises(P.PngfError):
        ctx.score_flips([0, 1], want_ports=True)
    ctx.close()


def test_pec_trace_capacity_completes_the_search(P):
    """A trace shorter than the run (here none at all) ends nothing early: the
    search completes with PNGF_ECAPACITY reported and the oracle's end state."""
    case = _case("fdfd64")
    b0 = W.random_design(case.n_d, 0)
    ref = O.dbs(O.Problem.from_case(case), b0, W.raster_order(case.n_d, 6), tau=1e-6, evaluator=O.evaluate_pec)
    for cap in (0, 5):
        ctx = P.DbsContext(case, precision=P.PNGF_PEC, tau=1e-6)
        ctx.factor(b0)
        if cap == 0:
            P.pngf_dbs_sweep(ctx.ctx, 6, None, None, None, 0, ctx.counters.data_ptr())
            assert ctx.sync() == P.PNGF_OK
            c = ctx.counters.cpu().numpy()
        else:
            c = ctx.dbs_sweep(6, trace_cap=cap)["counters"]
        assert c[0] == len(ref.accepted) and c[6] == P.PNGF_ECAPACITY
        assert np.array_equal(ctx.design(), ref.b)
        ctx.close()
