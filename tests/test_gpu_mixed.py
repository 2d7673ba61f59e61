"""Mixed-precision path (FP32 maintained inverse + FP64 decisions) through the C ABI.

Bars:
* right after the factor the scored state is FP64 (same as the FP64 path):
  candidate objectives within 1e-9 of the oracle;
* after kept flips the state follows the oracle's re-solves to FP32 accuracy
  amplified by the conditioning (1e-5 relative on the dielectric cases);
* DBS: when every oracle decision margin exceeds 1e-6 |f| (above the error of
  a mixed-precision score: FP32 rounding 6e-8 of the maintained inverse,
  amplified by the conditioning of M, ~1e-7 on these cases) the accepted
  sequence equals the oracle's, and the final S-parameters agree within 1e-4
  relative (the spec accuracy bar).
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


@pytest.fixture(scope="module")
def fdfd64():
    return W.get_case("fdfd64")


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def s_rel(case, o, o_ref):
    S = (np.asarray(o) - case.s_off) * case.s_scale
    Sr = (np.asarray(o_ref) - case.s_off) * case.s_scale
    return float(np.max(np.abs(S - Sr) / np.maximum(np.abs(Sr), 1e-3)))


def _ctx(P, case, **kw):
    kw.setdefault("precision", P.PNGF_MIXED)
    return P.DbsContext(case, **kw)


def test_mixed_factor_state_is_fp64(P, fdfd64):
    case = fdfd64
    b = W.random_design(case.n_d, 11)
    ctx = _ctx(P, case, delay_r=8, refresh_k=16)
    ctx.factor(b)
    st = ctx.state()
    v = case.dv * b
    Wr = O.maintained_inverse(case.G_dd, v)
    assert rel(st["diag"], np.diag(Wr)) < 1e-10
    assert rel(st["T"], O.port_projection(case.G_dd, case.G_od, v)) < 1e-10
    f_gpu = ctx.score_flips(np.arange(case.n_d))
    f_ref = O.candidate_objectives(O.Problem.from_case(case), b, np.arange(case.n_d))
    assert np.max(np.abs(f_gpu - f_ref) / np.abs(f_ref)) < 1e-9


@pytest.mark.parametrize("tensor_fold", [0, 1])
def test_mixed_refresh_restores_fp64_accuracy(P, fdfd64, tensor_fold):
    """A refresh (the double-float residual r = rhs - M y, then y += W (v r) in
    FP32) leaves e and T at FP64-level error for the current design, orders of
    magnitude below the FP32 drift the same kept flips leave without one.

    Best-improvement mode stops after exactly n_sweeps kept flips, and with
    delay_r = refresh_k = 16 the 16th kept flip is followed by a fold and a
    refresh, so the state read back is the refreshed one."""
    case = fdfd64
    b0 = W.random_design(case.n_d, 5)
    errs = {}
    for rk in (16, 0):
        ctx = _ctx(P, case, mode=P.PNGF_BEST_IMPROVEMENT, tau=1e-9, delay_r=16, refresh_k=rk,
                   tensor_fold=tensor_fold)
        ctx.factor(b0)
        cnt = ctx.dbs_sweep(16)["counters"]
        assert int(cnt[0]) == 16 and int(cnt[4]) == (1 if rk else 0)
        b = ctx.design()
        v = case.dv * b
        st = ctx.state()
        e_ref = O.solve_field(case.G_dd, case.c_d, v)
        T_ref = O.port_projection(case.G_dd, case.G_od, v)
        errs[rk] = max(rel(st["e"], e_ref), rel(st["T"], T_ref))
        ctx.close()
    print("state error after 16 kept flips: refreshed %.3e, not refreshed %.3e" % (errs[16], errs[0]))
    assert errs[16] < 1e-11
    assert errs[0] > 100 * errs[16]


@pytest.fixture(scope="module")
def fdfd256():
    return W.get_case("fdfd256")


@pytest.mark.parametrize("n_sub,n_ctas", [(997, 5), (1024, 7), (1501, 19), (4096, 19)])
def test_mixed_refresh_accuracy_across_grids(P, fdfd256, n_sub, n_ctas):
    """The refresh at ragged region sizes and several CTA counts, where the
    correction's work (the upper triangle of W row by row, two rows per warp;
    the active rows above each block of 32 columns) is dealt over the grid in
    snake order and the own rows gather the sums after a grid barrier: after
    16 kept flips, the 16th followed by a fold and a refresh, e and T are at
    FP64-level error against direct solves of the current design."""
    case = fdfd256 if n_sub == fdfd256.n_d else fdfd256.sub_case(np.arange(n_sub))
    b0 = W.random_design(case.n_d, 11)
    ctx = _ctx(P, case, mode=P.PNGF_BEST_IMPROVEMENT, tau=1e-9, delay_r=16, refresh_k=16, n_ctas=n_ctas)
    ctx.factor(b0)
    cnt = ctx.dbs_sweep(16)["counters"]
    assert int(cnt[0]) == 16 and int(cnt[4]) == 1
    b = ctx.design()
    v = case.dv * b
    st = ctx.state()
    err = max(rel(st["e"], O.solve_field(case.G_dd, case.c_d, v)),
              rel(st["T"], O.port_projection(case.G_dd, case.G_od, v)))
    print(f"n_d {case.n_d}, {n_ctas} CTAs: refreshed state error {err:.3e}")
    assert err < 1e-11
    ctx.close()


@pytest.mark.parametrize("n_accepts", [3, 8, 13])
def test_mixed_accepts_follow_resolves(P, fdfd64, n_accepts):
    """Standalone accepts across a flush (delay_r = 4)."""
    case = fdfd64
    b = W.random_design(case.n_d, 7)
    ctx = _ctx(P, case, delay_r=4, refresh_k=0)
    ctx.factor(b)
    rng = np.random.default_rng(n_accepts)
    for k in rng.choice(case.n_d, n_accepts, replace=False):
        ctx.accept_flip(int(k))
        b[k] ^= 1
    st = ctx.state()
    v = case.dv * b
    Wr = O.maintained_inverse(case.G_dd, v)
    ev = O.evaluate(O.Problem.from_case(case), b)
    assert rel(st["diag"], np.diag(Wr)) < 1e-5
    assert rel(st["e"], ev.e) < 1e-5
    assert rel(st["T"], O.port_projection(case.G_dd, case.G_od, v)) < 1e-5
    o, _ = ctx.eval_ports()
    assert s_rel(case, o, ev.o) < 1e-5
    assert np.array_equal(ctx.design(), b)
    # the scores after the accepts agree with re-solves to FP32-level accuracy
    f_gpu = ctx.score_flips(np.arange(0, case.n_d, 7))
    f_ref = O.candidate_objectives(O.Problem.from_case(case), b, np.arange(0, case.n_d, 7))
    assert np.max(np.abs(f_gpu - f_ref) / np.abs(f_ref)) < 1e-5


def _golden(name):
    with open(os.path.join(HERE, "golden", f"{name}.json")) as fh:
        return json.load(fh)


@pytest.mark.parametrize("name", ["fdfd64_first_raster", "fdfd64_first_shuffled", "fdfd64_best"])
@pytest.mark.parametrize("delay_r,refresh_k,tensor_fold", [(4, 8, 0), (16, 32, 0), (64, 0, 0), (32, 32, 1), (64, 64, 1)])
def test_mixed_dbs_matches_oracle(P, fdfd64, name, delay_r, refresh_k, tensor_fold):
    g = _golden(name)
    case = fdfd64
    sp = g["spec"]
    assert g["min_abs_margin"] > 1e-6 * abs(g["final_f"])  # decisions far from the score error
    b0 = W.random_design(case.n_d, sp["seed"])
    mode = P.PNGF_BEST_IMPROVEMENT if sp["mode"] == O.BEST_IMPROVEMENT else P.PNGF_FIRST_IMPROVEMENT
    ctx = _ctx(P, case, mode=mode, tau=g["tau"], delay_r=delay_r, refresh_k=refresh_k, tensor_fold=tensor_fold)
    ctx.factor(b0)
    order = None if sp["order"] == "raster" else W.shuffled_order(case.n_d, sp["n_sweeps"], seed=sp["seed"])
    res = ctx.dbs_sweep(sp["n_sweeps"], order=order)
    ref_k = [k for _, _, k, _ in g["accepted"]]
    assert [int(r[2]) for r in res["trace"]] == ref_k
    assert np.array_equal(ctx.design(), np.array(g["final_b"], np.uint8))
    o, _ = ctx.eval_ports()
    o_ref = np.array([complex(*z) for z in g["final_o"]])
    assert s_rel(case, o, o_ref) < 1e-4
    c = res["counters"]
    assert c[1] == g["n_evals"]
    assert c[5] == len(ref_k) // delay_r  # flushes


@pytest.mark.parametrize("mode", ["first", "best"])
def test_mixed_min_objective_matches_oracle(P, fdfd64, mode):
    """The minimised objective, f = sum_p w_p (1 - |S_p|)^2 (the insertion-loss
    form, w = (0, 1)), through the mixed path with folds and refreshes: the
    accepted sequence equals the oracle's (decision margins above 1e-5 |f| for
    this start) and the final S-parameters agree within 1e-4."""
    import dataclasses
    case = dataclasses.replace(fdfd64, obj_kind=W.OBJ_MIN_INSERTION_LOSS, obj_weights=np.array([0.0, 1.0]))
    p = O.Problem.from_case(case)
    b0 = W.random_design(case.n_d, 4)
    first = mode == "first"
    n_sweeps = 3 if first else 40
    order = np.tile(np.arange(case.n_d, dtype=np.int32), (n_sweeps, 1))
    ref = O.dbs(p, b0, order, tau=1e-9, mode=O.FIRST_IMPROVEMENT if first else O.BEST_IMPROVEMENT)
    assert ref.min_abs_margin > 1e-6 * abs(ref.f)
    ctx = _ctx(P, case, mode=P.PNGF_FIRST_IMPROVEMENT if first else P.PNGF_BEST_IMPROVEMENT, tau=1e-9,
               delay_r=16, refresh_k=32, tensor_fold=1)
    ctx.factor(b0)
    res = ctx.dbs_sweep(n_sweeps)
    assert [int(r[2]) for r in res["trace"]] == [k for _, _, k, _ in ref.accepted]
    assert np.array_equal(ctx.design(), ref.b)
    f_trace = np.array([fa for _, _, _, fa in ref.accepted])
    # relative to |f|, floored at 1e-6 of the run's largest f: the insertion loss
    # reaches exactly 0 (T21 = 1 at the empty design), where no relative bar applies
    floor = 1e-6 * np.max(np.abs(f_trace))
    assert np.max(np.abs(res["trace_f"] - f_trace) / np.maximum(np.abs(f_trace), floor)) < 1e-5
    o, _ = ctx.eval_ports()
    assert s_rel(case, o, ref.o) < 1e-4


def test_mixed_restore_replays(P, fdfd64):
    ctx = _ctx(P, fdfd64, delay_r=8, refresh_k=16)
    ctx.factor(W.random_design(fdfd64.n_d, 0))
    ctx.snapshot()
    r1 = ctx.dbs_sweep(3)
    ctx.restore()
    r2 = ctx.dbs_sweep(3)
    assert np.array_equal(r1["trace"], r2["trace"])
    assert np.array_equal(r1["trace_f"], r2["trace_f"])


@pytest.mark.parametrize("tensor_fold", [0, 1])
def test_mixed_vs_fp64_full_size(P, tensor_fold):
    """N_d = 4096 (the bench workload): the mixed run against the FP64 run and
    the oracle; S-parameters of the final design within 1e-4 relative."""
    case = W.get_case("fdfd256")
    b0 = W.random_design(case.n_d, 0)
    f64 = P.DbsContext(case, precision=P.PNGF_FP64, refresh_k=64)
    f64.factor(b0)
    r64 = f64.dbs_sweep(10)
    mix = _ctx(P, case, delay_r=64, refresh_k=64, tensor_fold=tensor_fold)
    mix.factor(b0)
    rmx = mix.dbs_sweep(10)
    k64 = [int(r[2]) for r in r64["trace"]]
    kmx = [int(r[2]) for r in rmx["trace"]]
    n_same = next((i for i, (x, y) in enumerate(zip(k64, kmx)) if x != y), min(len(k64), len(kmx)))
    print(f"fp64 accepts {len(k64)}, mixed {len(kmx)}, identical prefix {n_same}")
    p = O.Problem.from_case(case)
    ev = O.evaluate(p, mix.design())
    o, _ = mix.eval_ports()
    err = s_rel(case, o, ev.o)
    print(f"mixed final-design S error vs oracle {err:.2e}")
    assert err < 1e-4
    assert n_same >= min(100, len(k64))


@pytest.mark.parametrize("name,delay_r,n_acc", [("fdfd64", 32, 40), ("fdfd64", 64, 70), ("fdfd256", 64, 140)])
def test_tensor_fold_matches_cuda_core_fold(P, name, delay_r, n_acc):
    """The tcgen05 (3xTF32) fold of the delayed set against the FP32 CUDA-core
    fold, and both against the oracle, across several folds (ragged tiles on
    the 100-pixel region)."""
    case = W.get_case(name)
    b = W.random_design(case.n_d, 2)
    ctxs = []
    for tf in (0, 1):
        c = _ctx(P, case, delay_r=delay_r, refresh_k=0, tensor_fold=tf)
        c.factor(b)
        ctxs.append(c)
    rng = np.random.default_rng(5)
    pix = rng.choice(case.n_d, n_acc, replace=False)
    for k in pix:
        for c in ctxs:
            c.accept_flip(int(k))
        b[k] ^= 1
    s0, s1 = ctxs[0].state(), ctxs[1].state()
    for key in ("diag", "e", "T"):
        assert rel(s1[key], s0[key]) < 2e-6, key
    o0, _ = ctxs[0].eval_ports()
    o1, _ = ctxs[1].eval_ports()
    ev = O.evaluate(O.Problem.from_case(case), b)
    assert s_rel(case, o1, ev.o) < 1e-4
    assert s_rel(case, o1, o0) < 1e-5
    assert ctxs[1].sync() == 0


def test_mixed_sweep_rejects_grid_too_small(P, fdfd64):
    """More than 256 pixels per CTA of the persistent grid, or more delayed rows
    than the work area holds, is refused before any launch."""
    ctx = _ctx(P, fdfd64, delay_r=8, refresh_k=16, n_ctas=1)  # 100 pixels on one CTA: accepted
    ctx.factor(W.random_design(fdfd64.n_d, 0))
    ctx.dbs_sweep(1)
    big = W.get_case("fdfd128_metal")  # 1024 pixels
    ctx = _ctx(P, big, delay_r=8, refresh_k=16, n_ctas=3)  # 342 per CTA
    ctx.factor(W.random_design(big.n_d, 0))
    with pytest.raises(P.PngfError) as ei:
        ctx.dbs_sweep(1)
    assert ei.value.status == P.PNGF_EINVAL
    ctx = _ctx(P, big, delay_r=128, refresh_k=128, n_ctas=4)  # 256 per CTA x (128 + 8) delayed rows: 272 KB
    ctx.factor(W.random_design(big.n_d, 0))
    with pytest.raises(P.PngfError) as ei:
        ctx.dbs_sweep(1)
    assert ei.value.status == P.PNGF_EINVAL
