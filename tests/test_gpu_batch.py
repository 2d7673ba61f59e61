"""Batched DBS (many independent runs, one launch) through the C ABI.

Every run of a batch must follow the same trajectory as the same run done
alone with pngf_dbs_sweep (both FP64 on the FP64 path: the decisions are the
same FP64 comparisons), and the small runs are also checked against the CPU
oracle.  Ragged design regions: principal sub-blocks of one region's G, as
the batched workload of many random starts on one device uses them.
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


def _square_block(side_big, x0, side):
    return np.array([(x0 + i) * side_big + (x0 + j) for i in range(side) for j in range(side)])


def _runs(fdfd64):
    rng = np.random.default_rng(3)
    subs = [fdfd64, fdfd64.sub_case(_square_block(10, 1, 8)), fdfd64.sub_case(np.sort(rng.choice(100, 37, False))),
            fdfd64, fdfd64.sub_case(_square_block(10, 2, 6))]
    seeds = [0, 1, 2, 3, 4]
    return subs, seeds


@pytest.mark.parametrize("precision,mode,tensor_fold", [("fp64", "first", 0), ("fp64", "best", 0),
                                                        ("mixed", "first", 0), ("mixed", "first", 1)])
def test_batch_equals_solo_runs(P, precision, mode, tensor_fold):
    fdfd64 = W.get_case("fdfd64")
    subs, seeds = _runs(fdfd64)
    prec = P.PNGF_FP64 if precision == "fp64" else P.PNGF_MIXED
    md = P.PNGF_FIRST_IMPROVEMENT if mode == "first" else P.PNGF_BEST_IMPROVEMENT
    n_sweeps = 6 if mode == "first" else 200
    # FP64 without refresh: batch and solo runs do the same FP64 operations per
    # pixel, so they must agree bit for bit (the refresh sums in another order)
    kw = dict(precision=prec, mode=md, tau=1e-9, refresh_k=0 if precision == "fp64" else 16, delay_r=8,
              tensor_fold=tensor_fold)
    orders = [None, W.shuffled_order(64, n_sweeps, 5) if mode == "first" else None, None, None, None]
    solo = []
    for case, seed, order in zip(subs, seeds, orders):
        c = P.DbsContext(case, **kw)
        c.factor(W.random_design(case.n_d, seed))
        solo.append((c.dbs_sweep(n_sweeps, order=order), c.eval_ports(), c.design()))
        c.close()
    ctxs = []
    for case, seed in zip(subs, seeds):
        c = P.DbsContext(case, **kw)
        c.factor(W.random_design(case.n_d, seed))
        ctxs.append(c)
    batch = P.DbsBatch(ctxs)
    res = batch.dbs_sweep(n_sweeps, orders=orders)
    for i, (c, r) in enumerate(zip(ctxs, res)):
        s_res, (s_o, s_f), s_b = solo[i]
        assert [int(x[2]) for x in r["trace"]] == [int(x[2]) for x in s_res["trace"]], i
        if mode == "first":
            assert np.array_equal(r["trace"][:, :2], s_res["trace"][:, :2]), i
        tol = 0.0 if precision == "fp64" else 1e-5
        assert np.max(np.abs(r["trace_f"] - s_res["trace_f"]) / np.abs(s_res["trace_f"])) <= tol
        assert np.array_equal(r["counters"][:4], s_res["counters"][:4]), (i, r["counters"], s_res["counters"])
        o, f = c.eval_ports()
        assert rel(o, s_o) <= tol
        assert np.array_equal(c.design(), s_b)


def test_batch_refresh_matches_solo(P):
    """With the FP64 refresh on, batch and solo agree to rounding of the refresh sums."""
    fdfd64 = W.get_case("fdfd64")
    subs, seeds = _runs(fdfd64)
    kw = dict(refresh_k=16)
    solo, ctxs = [], []
    for case, seed in zip(subs, seeds):
        c = P.DbsContext(case, **kw)
        c.factor(W.random_design(case.n_d, seed))
        solo.append((c.dbs_sweep(6), c.eval_ports()))
        c.close()
        c = P.DbsContext(case, **kw)
        c.factor(W.random_design(case.n_d, seed))
        ctxs.append(c)
    res = P.DbsBatch(ctxs).dbs_sweep(6)
    for (s_res, (s_o, _)), c, r in zip(solo, ctxs, res):
        assert np.array_equal(r["trace"][:, :3], s_res["trace"][:, :3])
        assert np.max(np.abs(r["trace_f"] - s_res["trace_f"]) / np.abs(s_res["trace_f"])) < 1e-12
        assert rel(c.eval_ports()[0], s_o) < 1e-12


def test_batch_small_runs_match_oracle(P):
    """Sub-regions of the lossy-metal device, FP64, against the oracle's re-solves."""
    big = W.get_case("fdfd128_metal")
    cases = [big.sub_case(_square_block(32, 8, 16)), big.sub_case(_square_block(32, 12, 8))]
    ctxs = []
    for i, case in enumerate(cases):
        c = P.DbsContext(case, refresh_k=64)
        c.factor(W.random_design(case.n_d, 10 + i))
        ctxs.append(c)
    res = P.DbsBatch(ctxs).dbs_sweep(1)
    for i, (case, c, r) in enumerate(zip(cases, ctxs, res)):
        p = O.Problem.from_case(case)
        ref = O.dbs(p, W.random_design(case.n_d, 10 + i), W.raster_order(case.n_d, 1), tau=1e-9,
                    keep_margins=True)
        n_clean = 0
        for (_, _, m, f_before) in ref.margins:
            if abs(m) < 1e-9 * max(abs(f_before), 1e-30):
                break
            if m > 0:
                n_clean += 1
        got = [(int(x[0]), int(x[1]), int(x[2])) for x in r["trace"][:n_clean]]
        assert got == [(s, t, k) for s, t, k, _ in ref.accepted[:n_clean]]
        if n_clean == len(ref.accepted) and len(r["trace"]) == n_clean:
            o, _ = c.eval_ports()
            assert rel(o, ref.o) < 1e-9


def test_batch_rejects_mixed_contexts(P):
    fdfd64 = W.get_case("fdfd64")
    a = P.DbsContext(fdfd64)
    b = P.DbsContext(fdfd64, precision=P.PNGF_MIXED, delay_r=8, refresh_k=16)
    a.factor(W.random_design(100, 0))
    b.factor(W.random_design(100, 0))
    with pytest.raises(P.PngfError) as ei:
        P.DbsBatch([a, b]).dbs_sweep(1)
    assert ei.value.status == P.PNGF_EINVAL


def test_batch_queue_many_ragged_runs(P):
    """More runs than SMs, of four region sizes in mixed order: the runs go
    through the batch call's queue (largest region first, one CTA per SM taking
    the next run), and every run still ends bit for bit as the same run done
    alone, whatever the order in which the caller lists them."""
    fdfd64 = W.get_case("fdfd64")
    rng = np.random.default_rng(11)
    sizes = [100, 64, 37, 16]
    subs = {n: (fdfd64 if n == 100 else fdfd64.sub_case(np.sort(rng.choice(100, n, False)))) for n in sizes}
    n_runs = 176  # above the 152 SMs of the part
    spec = [(sizes[(7 * i) % 4], i) for i in range(n_runs)]
    kw = dict(precision=P.PNGF_FP64, tau=1e-9, refresh_k=0)
    solo = []
    for n, seed in spec:
        c = P.DbsContext(subs[n], **kw)
        c.factor(W.random_design(n, seed))
        r = c.dbs_sweep(3)
        solo.append(([int(x[2]) for x in r["trace"]], c.eval_ports()[0], c.design()))
        c.close()
    for perm in (np.arange(n_runs), rng.permutation(n_runs)):
        ctxs = [None] * n_runs
        for i in perm:
            n, seed = spec[i]
            c = P.DbsContext(subs[n], **kw)
            c.factor(W.random_design(n, seed))
            ctxs[i] = c
        res = P.DbsBatch([ctxs[i] for i in perm]).dbs_sweep(3)
        for pos, i in enumerate(perm):
            k_s, o_s, b_s = solo[i]
            assert [int(x[2]) for x in res[pos]["trace"]] == k_s, i
            o, _ = ctxs[i].eval_ports()
            assert np.array_equal(o, o_s) and np.array_equal(ctxs[i].design(), b_s), i
        for c in ctxs:
            c.close()
