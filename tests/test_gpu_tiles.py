"""Tile flips on one or several systems (pngf_dbs_sweep_tiles and friends)
against the CPU oracle's dbs_tiles / tile_candidate_objectives.

Bars as the single-pixel FP64 path: the accepted sequence equals the
oracle's exactly (FP64 decisions, every oracle margin above 1e-9 |F|),
combined objectives and port amplitudes within 1e-9 relative, the maintained
inverse after a kept tile within 1e-10 of M^-1 G at the new design (1e-9 on
lossy metal).
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


def _systems(P, names, b0, refresh_k=16, mode=None):
    cases = [W.get_case(n) for n in names]
    kw = dict(tau=1e-9, refresh_k=refresh_k)
    if mode is not None:
        kw["mode"] = mode
    ctxs = []
    for c in cases:
        cx = P.DbsContext(c, **kw)
        cx.factor(b0)
        ctxs.append(cx)
    return cases, ctxs


TILE_RUNS = {
    # name: (systems, tile layout, seed, order, mode, combine, sweeps)
    "square2x2": (["fdfd64"], "square", 0, "raster", O.FIRST_IMPROVEMENT, O.COMBINE_MEAN, 8),
    "mirror_tied": (["fdfd64"], "mirror", 1, "shuffled", O.FIRST_IMPROVEMENT, O.COMBINE_MEAN, 8),
    "square_best": (["fdfd64"], "square", 2, "raster", O.BEST_IMPROVEMENT, O.COMBINE_MEAN, 8),
    "three_freq_pixels_mean": (["fdfd64", "fdfd64_l19", "fdfd64_l21"], "pixel", 5, "raster", O.FIRST_IMPROVEMENT,
                               O.COMBINE_MEAN, 4),
    "three_freq_pixels_worst": (["fdfd64", "fdfd64_l19", "fdfd64_l21"], "pixel", 5, "raster", O.FIRST_IMPROVEMENT,
                                O.COMBINE_WORST, 4),
    "two_freq_tiles_worst": (["fdfd64", "fdfd64_l19"], "square", 6, "raster", O.FIRST_IMPROVEMENT,
                             O.COMBINE_WORST, 6),
}


def _tiles(kind):
    if kind == "square":
        return W.square_tiles(10, 10, 2)
    if kind == "mirror":
        return W.mirror_tied_tiles(10, 10, 2)
    return np.arange(100, dtype=np.int32)[:, None]


@pytest.mark.parametrize("run", sorted(TILE_RUNS))
def test_tile_search_matches_oracle(P, run):
    names, layout, seed, order_kind, mode, combine, sweeps = TILE_RUNS[run]
    tiles = _tiles(layout)
    n_t = len(tiles)
    order = W.raster_order(n_t, sweeps) if order_kind == "raster" else W.shuffled_order(n_t, sweeps, seed=4)
    b0 = W.random_design(100, seed)
    cases, ctxs = _systems(P, names, b0, mode=mode)
    ref = O.dbs_tiles([O.Problem.from_case(c) for c in cases], b0, tiles, order, tau=1e-9, mode=mode,
                      combine=combine)
    assert ref.min_abs_margin > 1e-9 * abs(ref.f)
    ts = P.TileSearch(ctxs, tiles, combine=combine)
    res = ts.dbs_sweep(sweeps, order=order if order_kind == "shuffled" else None)
    got = [tuple(int(x) for x in r[:3]) for r in res["trace"]]
    assert got == [tuple(a[:3]) for a in ref.accepted]
    f_ref = np.array([a[3] for a in ref.accepted])
    assert np.max(np.abs(res["trace_f"] - f_ref)) <= 1e-9 * np.max(np.abs(f_ref))
    assert res["counters"][1] == ref.n_evals and res["counters"][2] == ref.sweeps_done
    for cx, o_ref in zip(ctxs, ref.o_all):
        assert np.array_equal(cx.design(), ref.b)
        o, _ = cx.eval_ports()
        assert rel(o, o_ref) < 1e-9
    for cx in ctxs:
        cx.close()


@pytest.mark.parametrize("names,layout,combine", [(["fdfd64", "fdfd64_l21"], "mirror", O.COMBINE_MEAN),
                                                  (["fdfd128_metal"], "square16", O.COMBINE_MEAN)])
def test_score_tiles_parity(P, names, layout, combine):
    if layout == "square16":
        tiles = W.square_tiles(32, 32, 2)[::8]  # 32 of the 256 2 x 2 tiles of the 32 x 32 region
        n_d = 1024
    else:
        tiles = _tiles(layout)
        n_d = 100
    b0 = W.random_design(n_d, 9)
    cases, ctxs = _systems(P, names, b0)
    ts = P.TileSearch(ctxs, tiles, combine=combine)
    F, fs = ts.score(per_system=True)
    probs = [O.Problem.from_case(c) for c in cases]
    ref = O.tile_candidate_objectives(probs, b0, tiles, combine)
    tol = 5e-9 if names == ["fdfd128_metal"] else 1e-9
    assert np.max(np.abs(F - ref) / np.abs(ref)) < tol
    for s, p in enumerate(probs):
        ref_s = np.array([O.evaluate(p, O.flip_tile(b0, t)).f for t in tiles])
        assert np.max(np.abs(fs[:, s] - ref_s) / np.abs(ref_s)) < tol
    for cx in ctxs:
        cx.close()


@pytest.mark.parametrize("names,tile", [(["fdfd64"], 7), (["fdfd64", "fdfd64_l19"], 12),
                                        (["fdfd128_metal"], 100)])
def test_accept_tile_updates_the_inverse(P, names, tile):
    n_d = 1024 if names == ["fdfd128_metal"] else 100
    side = 32 if n_d == 1024 else 10
    tiles = W.mirror_tied_tiles(side, side, 2)
    b0 = W.random_design(n_d, 3)
    cases, ctxs = _systems(P, names, b0)
    ts = P.TileSearch(ctxs, tiles)
    ts.accept(tile)
    b1 = O.flip_tile(b0, tiles[tile])
    tol = 1e-9 if n_d == 1024 else 1e-10
    for c, cx in zip(cases, ctxs):
        st = cx.state(with_W=True)
        v = c.dv * b1
        Wr = O.maintained_inverse(c.G_dd, v)
        iu = np.triu_indices(n_d)
        assert rel(st["W"][iu], Wr[iu]) < tol
        assert rel(st["diag"], np.diag(Wr)) < tol
        ev = O.evaluate(O.Problem.from_case(c), b1)
        assert rel(st["e"], ev.e) < tol
        assert rel(st["T"], O.port_projection(c.G_dd, c.G_od, v)) < tol
        assert rel(cx.eval_ports()[0], ev.o) < tol
        assert np.array_equal(cx.design(), b1)
    for cx in ctxs:
        cx.close()


def test_tile_arguments_are_checked(P):
    b0 = W.random_design(100, 0)
    cases, ctxs = _systems(P, ["fdfd64"], b0)
    with pytest.raises(P.PngfError):
        P.TileSearch(ctxs, np.zeros((4, 17), np.int32))  # tile_m above PNGF_TILE_MAX
    mixed = P.DbsContext(cases[0], precision=P.PNGF_MIXED, delay_r=8, refresh_k=16)
    mixed.factor(b0)
    with pytest.raises(P.PngfError):
        P.TileSearch([ctxs[0], mixed], W.square_tiles(10, 10, 2)).score()
    # an out-of-range pixel in a tile latches PNGF_EINVAL on the device
    bad = W.square_tiles(10, 10, 2).copy()
    bad[3, 1] = 100
    ts = P.TileSearch(ctxs, bad)
    ts.dbs_sweep(2, sync=False)
    assert ctxs[0].sync() == P.PNGF_EINVAL
    mixed.close()
    ctxs[0].close()


def test_tile_trace_capacity_completes_the_search(P):
    tiles = _tiles("square")
    b0 = W.random_design(100, 0)
    cases, ctxs = _systems(P, ["fdfd64"], b0)
    ref = O.dbs_tiles([O.Problem.from_case(cases[0])], b0, tiles, W.raster_order(len(tiles), 8), tau=1e-9)
    ts = P.TileSearch(ctxs, tiles)
    res = ts.dbs_sweep(8, trace_cap=3)
    assert res["counters"][0] == len(ref.accepted) and res["counters"][6] == P.PNGF_ECAPACITY
    assert np.array_equal(ctxs[0].design(), ref.b)
    ctxs[0].close()
