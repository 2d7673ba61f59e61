"""Parity of the CUDA path (through the C ABI) with the CPU oracle -- FP64 path.

Bars (written here, derived in the design notes):
* factor / maintained state: relative max error <= 1e-10 on the well-
  conditioned cases, 1e-9 on the lossy-metal case (cond(M) ~ 5e6, so two
  correct FP64 solvers differ by ~cond * eps);
* candidate objectives: relative error <= 1e-9;
* DBS: the accepted-flip sequence equals the oracle's exactly (FP64 on both
  sides decides every flip) while the oracle's decision margins exceed
  1e-9 |f|; port amplitudes within 1e-9 relative.
"""
import json
import os

import numpy as np
import pytest

from paper_2501_18054_gb300 import workloads as W
import oracle as O

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def P():
    from paper_2501_18054_gb300 import build as B
    B.build()
    from paper_2501_18054_gb300 import pngf
    return pngf


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module")
def fdfd64():
    return W.get_case("fdfd64")


@pytest.fixture(scope="module")
def metal128():
    return W.get_case("fdfd128_metal")


def _ctx(P, case, **kw):
    return P.DbsContext(case, **kw)


def _ragged(fdfd64, n):
    rng = np.random.default_rng(n)
    return fdfd64.sub_case(np.sort(rng.choice(fdfd64.n_d, n, replace=False)), name=f"fdfd64_sub{n}")


@pytest.mark.parametrize("which", ["fdfd64", "metal128", "ragged97", "ragged33", "single"])
def test_factor_state_parity(P, fdfd64, metal128, which):
    case = {"fdfd64": fdfd64, "metal128": metal128}.get(which)
    if which.startswith("ragged"):
        case = _ragged(fdfd64, int(which[6:]))
    if which == "single":
        case = fdfd64.sub_case([44])
    tol = 1e-9 if which == "metal128" else 1e-10
    b = W.random_design(case.n_d, 11) if case.n_d > 1 else np.ones(1, np.uint8)
    ctx = _ctx(P, case)
    ctx.factor(b)
    st = ctx.state(with_W=True)
    p = O.Problem.from_case(case)
    v = case.dv * b
    Wr = O.maintained_inverse(case.G_dd, v)
    Tr = O.port_projection(case.G_dd, case.G_od, v)
    ev = O.evaluate(p, b)
    assert rel(st["W"], Wr) < tol
    assert rel(st["diag"], np.diag(Wr)) < tol
    assert rel(st["e"], ev.e) < tol
    assert rel(st["T"], Tr) < tol
    o, f = ctx.eval_ports()
    assert rel(o, ev.o) < tol
    assert abs(f - ev.f) <= tol * abs(ev.f)
    assert np.array_equal(ctx.design(), b)


def test_empty_design_gives_G(P, fdfd64):
    ctx = _ctx(P, fdfd64)
    ctx.factor(np.zeros(fdfd64.n_d, np.uint8))
    st = ctx.state(with_W=True)
    assert rel(st["W"], fdfd64.G_dd) < 1e-14
    o, _ = ctx.eval_ports()
    assert rel(o, fdfd64.c_o) < 1e-14


@pytest.mark.parametrize("which", ["fdfd64", "metal128"])
def test_score_flips_parity(P, fdfd64, metal128, which):
    case = fdfd64 if which == "fdfd64" else metal128
    b = W.random_design(case.n_d, 5)
    ctx = _ctx(P, case)
    ctx.factor(b)
    rng = np.random.default_rng(1)
    cand = np.arange(case.n_d) if case.n_d <= 128 else np.sort(rng.choice(case.n_d, 96, replace=False))
    f_gpu, o_gpu = ctx.score_flips(cand, want_ports=True)
    p = O.Problem.from_case(case)
    f_ref = O.candidate_objectives(p, b, cand)
    o_ref = O.candidate_ports(p, b, cand)
    # lossy metal: cond(M) ~ 5e6 and |S21|^2 ~ 1e-9, so two correct FP64 solvers
    # differ by ~cond * eps ~ 5e-10 in each amplitude and twice that in |S|^2
    tol = 1e-9 if which == "fdfd64" else 5e-9
    assert np.max(np.abs(f_gpu - f_ref) / np.abs(f_ref)) < tol
    assert rel(o_gpu, o_ref) < tol


def test_accept_flip_parity(P, fdfd64):
    case = fdfd64
    b = W.random_design(case.n_d, 7)
    ctx = _ctx(P, case)
    ctx.factor(b)
    for k in (3, 50, 99, 0, 51):
        ctx.accept_flip(k)
        b[k] ^= 1
    st = ctx.state(with_W=True)
    v = case.dv * b
    Wr = O.maintained_inverse(case.G_dd, v)
    iu = np.triu_indices(case.n_d)
    assert rel(st["W"][iu], Wr[iu]) < 1e-11
    assert rel(st["diag"], np.diag(Wr)) < 1e-11
    ev = O.evaluate(O.Problem.from_case(case), b)
    assert rel(st["e"], ev.e) < 1e-11
    assert rel(st["T"], O.port_projection(case.G_dd, case.G_od, v)) < 1e-11
    o, f = ctx.eval_ports()
    assert rel(o, ev.o) < 1e-11
    assert np.array_equal(ctx.design(), b)


def _golden(name):
    with open(os.path.join(HERE, "golden", f"{name}.json")) as fh:
        return json.load(fh)


def _order(g, n_d):
    sp = g["spec"]
    if sp["order"] == "raster":
        return None, W.raster_order(n_d, sp["n_sweeps"])
    o = W.shuffled_order(n_d, sp["n_sweeps"], seed=sp["seed"])
    return o, o


@pytest.mark.parametrize("name", ["fdfd64_first_raster", "fdfd64_first_shuffled", "fdfd64_best"])
@pytest.mark.parametrize("refresh_k", [0, 16])
def test_dbs_trajectory_matches_golden(P, fdfd64, name, refresh_k):
    g = _golden(name)
    case = fdfd64
    sp = g["spec"]
    b0 = W.random_design(case.n_d, sp["seed"])
    mode = P.PNGF_BEST_IMPROVEMENT if sp["mode"] == O.BEST_IMPROVEMENT else P.PNGF_FIRST_IMPROVEMENT
    ctx = _ctx(P, case, mode=mode, tau=g["tau"], refresh_k=refresh_k)
    ctx.factor(b0)
    order_dev, _ = _order(g, case.n_d)
    res = ctx.dbs_sweep(sp["n_sweeps"], order=order_dev)
    assert g["min_abs_margin"] > 1e-9 * abs(g["final_f"])  # no near-tie: the sequence is unique
    acc_ref = [(s, t, k) for s, t, k, _ in g["accepted"]]
    tr = res["trace"]
    if mode == P.PNGF_FIRST_IMPROVEMENT:
        acc_gpu = [tuple(int(x) for x in r[:3]) for r in tr]
    else:
        acc_ref = [k for _, _, k in acc_ref]
        acc_gpu = [int(r[2]) for r in tr]
    assert acc_gpu == acc_ref
    f_ref = np.array([f for *_, f in g["accepted"]])
    assert np.max(np.abs(res["trace_f"] - f_ref) / np.abs(f_ref)) < 1e-9
    c = res["counters"]
    assert c[0] == len(acc_ref) and c[1] == g["n_evals"] and c[2] == g["sweeps_done"]
    assert np.array_equal(ctx.design(), np.array(g["final_b"], np.uint8))
    o, f = ctx.eval_ports()
    o_ref = np.array([complex(*z) for z in g["final_o"]])
    assert rel(o, o_ref) < 1e-9
    # and against a live oracle evaluation of the final design
    ev = O.evaluate(O.Problem.from_case(case), ctx.design())
    assert rel(o, ev.o) < 1e-9


def test_dbs_metal_prefix_and_validity(P, metal128):
    """Lossy metal (cond ~ 5e6): the sequence matches the oracle's up to its first
    near-tie (|margin| < 1e-9 |f|); kept flips past it are re-verified by
    independent re-solves; ports within 1e-9 relative."""
    case = metal128
    p = O.Problem.from_case(case)
    b0 = W.random_design(case.n_d, 0)
    ctx = _ctx(P, case, refresh_k=64)
    ctx.factor(b0)
    res = ctx.dbs_sweep(1)
    tr = res["trace"]
    assert len(tr) > 50
    ref = O.dbs(p, b0, W.raster_order(case.n_d, 1), tau=1e-9, keep_margins=True)
    # number of oracle accepts before its first ambiguous decision
    n_clean = 0
    for (_, _, m, f_before) in ref.margins:
        if abs(m) < 1e-9 * max(abs(f_before), 1e-30):
            break
        if m > 0:
            n_clean += 1
    assert n_clean >= 10
    gpu = [(int(r[0]), int(r[1]), int(r[2])) for r in tr[:n_clean]]
    assert gpu == [(s, t, k) for s, t, k, _ in ref.accepted[:n_clean]]
    b = b0.copy()
    steps = set(np.linspace(n_clean, len(tr) - 1, 8).astype(int).tolist())
    for i, r in enumerate(tr):
        k = int(r[2])
        if i in steps:
            f0 = O.evaluate(p, b).f
            b1 = b.copy(); b1[k] ^= 1
            f1 = O.evaluate(p, b1).f
            assert f1 - f0 > (1e-9 - 1e-8) * abs(f0)  # an improvement, up to the ambiguity band
        b[k] ^= 1
    o, _ = ctx.eval_ports()
    assert rel(o, O.evaluate(p, ctx.design()).o) < 1e-9


def test_restore_replays_the_same_run(P, fdfd64):
    case = fdfd64
    ctx = _ctx(P, case)
    ctx.factor(W.random_design(case.n_d, 0))
    ctx.snapshot()
    r1 = ctx.dbs_sweep(3)
    ctx.restore()
    r2 = ctx.dbs_sweep(3)
    assert np.array_equal(r1["trace"], r2["trace"])
    assert np.array_equal(r1["trace_f"], r2["trace_f"])


def test_trace_capacity_and_zero_sweeps(P, fdfd64):
    case = fdfd64
    ctx = _ctx(P, case)
    ctx.factor(W.random_design(case.n_d, 0))
    ctx.snapshot()
    r0 = ctx.dbs_sweep(0)
    assert r0 is None or r0["counters"][0] == 0
    res = ctx.dbs_sweep(3, trace_cap=10)
    c = res["counters"]
    g = _golden("fdfd64_first_raster")
    assert len(g["accepted"]) > 10
    assert c[0] == len(g["accepted"]) and c[6] == P.PNGF_ECAPACITY and len(res["trace"]) == 10
    assert np.array_equal(ctx.design(), np.array(g["final_b"], np.uint8))


def test_status_errors(P, fdfd64):
    ctx = _ctx(P, fdfd64)
    with pytest.raises(P.PngfError) as ei:
        ctx.score_flips([0, 1])
    assert ei.value.status == P.PNGF_ENOTFACTORED
    ctx.factor(W.random_design(fdfd64.n_d, 0))
    with pytest.raises(P.PngfError) as ei:
        ctx.accept_flip(fdfd64.n_d)
    assert ei.value.status == P.PNGF_EINVAL
    f = ctx.score_flips([-1, 5])
    assert np.isnan(f[0]) and np.isfinite(f[1])


def test_full_size_fdfd256_sampled(P):
    """N_d = 4096 in the bench's launch configuration: final ports against one
    oracle solve, and a sample of kept flips re-verified by re-solves."""
    case = W.get_case("fdfd256")
    p = O.Problem.from_case(case)
    b0 = W.random_design(case.n_d, 0)
    ctx = _ctx(P, case, refresh_k=64)
    ctx.factor(b0)
    res = ctx.dbs_sweep(1)
    tr = res["trace"]
    assert res["counters"][1] == case.n_d
    assert 100 < len(tr) < case.n_d
    o, _ = ctx.eval_ports()
    b_end = ctx.design()
    assert rel(o, O.evaluate(p, b_end).o) < 1e-9
    # re-verify 3 kept flips: the design before each is b0 with the earlier flips applied
    b = b0.copy()
    pick = {5, len(tr) // 2, len(tr) - 1}
    for i, r in enumerate(tr):
        k = int(r[2])
        if i in pick:
            f0 = O.evaluate(p, b).f
            b1 = b.copy(); b1[k] ^= 1
            f1 = O.evaluate(p, b1).f
            assert f1 - f0 > 1e-9 * abs(f0)
            assert abs(res["trace_f"][i] - f1) < 1e-9 * abs(f1)
        b[k] ^= 1
    assert np.array_equal(b, b_end)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_invalid_order_is_rejected_on_device(P, fdfd64, precision):
    """An out-of-range visiting-order entry latches PNGF_EINVAL (never used as an index)."""
    kw = {} if precision == "fp64" else dict(precision=P.PNGF_MIXED, delay_r=8, refresh_k=16)
    ctx = _ctx(P, fdfd64, **kw)
    ctx.factor(W.random_design(fdfd64.n_d, 0))
    order = W.raster_order(fdfd64.n_d, 2)
    order[1, 17] = fdfd64.n_d + 5  # second sweep holds a bad entry
    with pytest.raises(P.PngfError) as ei:
        ctx.dbs_sweep(2, order=order)
    assert ei.value.status == P.PNGF_EINVAL
    # the context stays usable: a valid call afterwards succeeds
    res = ctx.dbs_sweep(1)
    assert res["counters"][6] in (P.PNGF_OK, P.PNGF_ECAPACITY)
