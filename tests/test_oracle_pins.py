"""Pins of the CPU oracle to things other than itself (CPU only).

* the reduced system against a direct sparse solve of the full modified FDFD
  structure (the paper's own accuracy check, Supplementary Note 8: the PNGF
  result agrees with the full solver to ~10 digits in double precision);
* the one-pixel closed form and the zero-contrast special case;
* brute-force enumeration of every design of a tiny region: the end state of
  the oracle's DBS is one-flip locally optimal, its trajectory only improves,
  and BEST mode takes the enumerated best neighbour every step;
* planted mistakes in the oracle are caught by these pins.
"""
import itertools

import numpy as np
import pytest

from paper_2501_18054_gb300 import workloads as W
import oracle as O


@pytest.fixture(scope="module")
def fdfd64():
    return W.make_fdfd_case("fdfd64")


@pytest.fixture(scope="module")
def metal128():
    return W.make_fdfd_case("fdfd128_metal")


def _full_structure(case, b):
    spec = W.SPECS[case.name]
    eps = W._eps_grid(spec)
    x0, y0, dx, dy = spec.design
    eps[x0:x0 + dx, y0:y0 + dy] = np.where(np.asarray(b).reshape(dx, dy) == 1, spec.eps_on, spec.eps_off)
    E, o = W.solve_full(spec, eps)
    return E[W._design_nodes(spec)], o


@pytest.mark.parametrize("name,seed", [("fdfd64", 3), ("fdfd64", 4), ("fdfd128_metal", 3)])
def test_reduced_system_equals_full_fdfd(name, seed, fdfd64, metal128):
    case = fdfd64 if name == "fdfd64" else metal128
    b = W.random_design(case.n_d, seed)
    ev = O.evaluate(O.Problem.from_case(case), b)
    e_full, o_full = _full_structure(case, b)
    assert np.max(np.abs(ev.e - e_full)) <= 1e-10 * np.max(np.abs(e_full))
    assert np.max(np.abs(ev.o - o_full)) <= 1e-10 * np.max(np.abs(o_full))


def test_one_pixel_closed_form(fdfd64):
    s = fdfd64.sub_case([57])
    p = O.Problem.from_case(s)
    ev = O.evaluate(p, np.array([1], np.uint8))
    g, c, v = s.G_dd[0, 0], s.c_d[0], s.dv[0]
    e = c / (1.0 - g * v)
    assert abs(ev.e[0] - e) <= 1e-15 * abs(e)
    o = s.c_o + s.G_od[:, 0] * v * e
    assert np.max(np.abs(ev.o - o)) <= 1e-15 * np.max(np.abs(o))


def test_zero_contrast_leaves_the_incident_field(fdfd64):
    p = O.Problem.from_case(fdfd64)
    p.dv = np.zeros_like(p.dv)
    ev = O.evaluate(p, W.random_design(fdfd64.n_d, 1))
    assert np.array_equal(ev.o, fdfd64.c_o)
    assert np.array_equal(ev.e, fdfd64.c_d)


def test_empty_design_is_the_incident_field(fdfd64):
    ev = O.evaluate(O.Problem.from_case(fdfd64), np.zeros(fdfd64.n_d, np.uint8))
    assert np.array_equal(ev.o, fdfd64.c_o)


def test_objectives():
    S = np.array([0.6 + 0.0j, 0.0 + 0.8j])
    assert O.objective(S, O.OBJ_MAX_WEIGHTED_POWER, np.array([0.0, 1.0])) == pytest.approx(0.64, abs=1e-15)
    assert O.objective(S, O.OBJ_MIN_INSERTION_LOSS, np.array([0.0, 1.0])) == pytest.approx(0.04, abs=1e-15)
    assert O.improvement(2.0, 1.0, O.OBJ_MAX_WEIGHTED_POWER) == 1.0
    assert O.improvement(2.0, 1.0, O.OBJ_MIN_INSERTION_LOSS) == -1.0


def _tiny(fdfd64, n_pix=12):
    # a 3 x 4 block in the middle of the 10 x 10 region (pixels k = 10*x + y)
    idx = [10 * x + y for x in range(3, 6) for y in range(3, 7)][:n_pix]
    return fdfd64.sub_case(idx)


def _enumerate(p):
    n = p.n_d
    fs = np.empty(2 ** n)
    for m in range(2 ** n):
        b = np.array([(m >> i) & 1 for i in range(n)], np.uint8)
        fs[m] = O.evaluate(p, b).f
    return fs


def _code(b):
    return int(sum(int(x) << i for i, x in enumerate(b)))


@pytest.fixture(scope="module")
def tiny(fdfd64):
    s = _tiny(fdfd64)
    p = O.Problem.from_case(s)
    return s, p, _enumerate(p)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_dbs_end_state_is_locally_optimal(tiny, seed):
    s, p, fs = tiny
    b0 = W.random_design(s.n_d, seed)
    tau = 1e-9
    res = O.dbs(p, b0, W.raster_order(s.n_d, 50), tau=tau)
    assert res.sweeps_done < 50  # converged
    f_end = fs[_code(res.b)]
    assert res.f == f_end
    for k in range(s.n_d):
        nb = res.b.copy(); nb[k] ^= 1
        assert fs[_code(nb)] - f_end <= tau * abs(f_end)
    # the trajectory only improves, and each kept flip is the first improving one in order
    f = fs[_code(b0)]
    b = b0.copy()
    last = (-1, -1)
    for (sw, t, k, f_after) in res.accepted:
        assert (sw, t) > last
        last = (sw, t)
        b[k] ^= 1
        assert f_after == fs[_code(b)] and f_after > f + tau * abs(f)
        f = f_after
    assert fs.max() >= f_end


@pytest.mark.parametrize("seed", [0, 5])
def test_dbs_best_mode_takes_the_best_neighbour(tiny, seed):
    s, p, fs = tiny
    b = W.random_design(s.n_d, seed)
    res = O.dbs(p, b, W.raster_order(s.n_d, 100), tau=1e-9, mode=O.BEST_IMPROVEMENT)
    for (_, _, k, f_after) in res.accepted:
        nbr = []
        for j in range(s.n_d):
            nb = b.copy(); nb[j] ^= 1
            nbr.append(fs[_code(nb)])
        assert k == int(np.argmax(nbr))
        b[k] ^= 1
        assert f_after == fs[_code(b)]


def test_dbs_shuffled_order_visits_every_pixel(tiny):
    s, p, fs = tiny
    order = W.shuffled_order(s.n_d, 40, seed=3)
    res = O.dbs(p, W.random_design(s.n_d, 9), order, tau=1e-9)
    for (sw, t, k, _) in res.accepted:
        assert order[sw, t] == k
    f_end = fs[_code(res.b)]
    for k in range(s.n_d):
        nb = res.b.copy(); nb[k] ^= 1
        assert fs[_code(nb)] - f_end <= 1e-9 * abs(f_end)


def test_dbs_counts_every_visited_position(fdfd64):
    s = _tiny(fdfd64, 8)
    p = O.Problem.from_case(s)
    res = O.dbs(p, W.random_design(8, 2), W.raster_order(8, 20), tau=1e-9)
    assert res.n_evals == res.sweeps_done * 8
    res2 = O.dbs(p, W.random_design(8, 2), W.raster_order(8, 20), tau=1e-9, max_evals=5)
    assert res2.n_evals == 5


def test_maintained_quantities_definitions(fdfd64):
    """W = M^-1 G and T = G_od (I + V W) against their defining systems."""
    s = _tiny(fdfd64)
    b = W.random_design(s.n_d, 1)
    v = s.dv * b
    M = O.system_matrix(s.G_dd, v)
    Wm = O.maintained_inverse(s.G_dd, v)
    assert np.max(np.abs(M @ Wm - s.G_dd)) < 1e-13
    T = O.port_projection(s.G_dd, s.G_od, v)
    # T M^T = G_od (M^-T = I + V W since W is symmetric)
    assert np.max(np.abs(T @ M.T - s.G_od)) < 1e-13
    assert np.max(np.abs(Wm - Wm.T)) < 1e-13


def test_planted_mistakes_are_caught(fdfd64, monkeypatch):
    """A plausible slip in the oracle fails the full-structure pin."""
    case = fdfd64
    b = W.random_design(case.n_d, 3)
    e_full, o_full = _full_structure(case, b)
    p = O.Problem.from_case(case)
    plants = {
        "sign of the contrast term": lambda G, v: np.eye(G.shape[0], dtype=complex) + G * v[None, :],
        "transposed contrast": lambda G, v: np.eye(G.shape[0], dtype=complex) - G * v[:, None],
        "dropped identity": lambda G, v: -G * v[None, :] + 1e-3 * np.eye(G.shape[0]),
    }
    for what, bad in plants.items():
        monkeypatch.setattr(O.pngf_oracle, "system_matrix", bad)
        ev = O.evaluate(p, b)
        assert np.max(np.abs(ev.o - o_full)) > 1e-6 * np.max(np.abs(o_full)), what
    monkeypatch.undo()
    monkeypatch.setattr(O.pngf_oracle, "port_amplitudes", lambda God, co, v, e: co + God @ e)
    ev = O.evaluate(p, b)
    assert np.max(np.abs(ev.o - o_full)) > 1e-6 * np.max(np.abs(o_full)), "dropped V in ports"


def _full_structure_S(case, b):
    """S-parameters of design b from direct sparse solves of full structures only.

    The definition is applied to full-solve port amplitudes, independently of
    the reduced system and of the oracle's affine map:
      free-space line ports ("incident"): S11 = (o_1 - o_1^empty)/o_1^empty and
        T21 = o_2/o_2^empty, the empty design's fields as the incident wave;
      waveguide ports ("reference"): S11 = (o_1 - a_1)/a_1 and S21 = o_2/a_2,
        a = the same source's mode amplitudes in the unbroken guide.
    """
    spec = W.SPECS[case.name]
    _, o = _full_structure(case, b)
    if spec.norm == "incident":
        _, a = _full_structure(case, np.zeros(case.n_d, np.uint8))
    else:
        _, a = W.solve_full(spec, W._eps_grid(spec, with_slab_through_design=True))
    return np.array([(o[0] - a[0]) / a[0]] + [o[p] / a[p] for p in range(1, len(o))])


@pytest.mark.parametrize("name,seed", [("fdfd64", 3), ("fdfd64", 8), ("fdfd128_metal", 5)])
def test_s_params_equal_full_structure(name, seed, fdfd64, metal128):
    """The oracle's S (evaluate, then the affine map) equals S from full solves."""
    case = fdfd64 if name == "fdfd64" else metal128
    b = W.random_design(case.n_d, seed)
    S = O.evaluate(O.Problem.from_case(case), b).S
    S_full = _full_structure_S(case, b)
    assert np.max(np.abs(S - S_full)) <= 1e-10 * max(1.0, np.max(np.abs(S_full)))
    # the configured objective of the free-space case is |T21|^2 = |o_2/o_2^empty|^2
    if name == "fdfd64":
        assert O.Problem.from_case(case).obj_weights.tolist() == [0.0, 1.0]
        f = O.evaluate(O.Problem.from_case(case), b).f
        assert abs(f - abs(S_full[1]) ** 2) <= 1e-10 * abs(f)


def test_planted_s_param_mistakes_are_caught(fdfd64, metal128, monkeypatch):
    """A plausible slip in the S map fails the full-structure S pin on some case."""
    cases = [(fdfd64, 3), (metal128, 5)]
    full = [_full_structure_S(c, W.random_design(c.n_d, s)) for c, s in cases]
    plants = {
        "offset after the scale": lambda o, off, sc: o * sc - off,
        "divided by the scale": lambda o, off, sc: (o - off) / sc,
        "offset added": lambda o, off, sc: (o + off) * sc,
        "offset on the other port": lambda o, off, sc: (o - off[::-1]) * sc,
        "scale of the other port": lambda o, off, sc: (o - off) * sc[::-1],
        "conjugated scale": lambda o, off, sc: (o - off) * np.conj(sc),
    }
    for what, bad in plants.items():
        monkeypatch.setattr(O.pngf_oracle, "s_params", bad)
        worst = 0.0
        for (c, s), Sf in zip(cases, full):
            S = O.evaluate(O.Problem.from_case(c), W.random_design(c.n_d, s)).S
            worst = max(worst, np.max(np.abs(S - Sf)) / np.max(np.abs(Sf)))
        assert worst > 1e-6, what
    monkeypatch.undo()


def _grad_fd(p, rho, ms, h=1e-5):
    out = []
    for m in ms:
        r1, r2 = rho.copy(), rho.copy()
        r1[m] += h
        r2[m] -= h
        out.append((O.evaluate(p, r1).f - O.evaluate(p, r2).f) / (2 * h))
    return np.array(out)


@pytest.mark.parametrize("kind", [O.OBJ_MAX_WEIGHTED_POWER, O.OBJ_MIN_INSERTION_LOSS])
@pytest.mark.parametrize("fractional", [False, True])
def test_gradient_equals_finite_differences(fdfd64, kind, fractional):
    """objective_gradient equals central differences of the pinned evaluate
    at a binary and at a fractional density (v = dv * rho)."""
    p = O.Problem.from_case(fdfd64)
    p.obj_kind = kind
    rng = np.random.default_rng(7)
    rho = W.random_design(fdfd64.n_d, 4).astype(np.float64)
    if fractional:
        rho = rng.random(fdfd64.n_d)
    g = O.objective_gradient(p, rho)
    ms = rng.choice(fdfd64.n_d, 12, replace=False)
    fd = _grad_fd(p, rho, ms)
    assert np.max(np.abs(g[ms] - fd)) <= 1e-6 * np.max(np.abs(fd))
    assert np.max(np.abs(fd)) > 1e-3


def test_gradient_one_pixel_closed_form(fdfd64):
    """N_d = 1: S(rho) = (c_o + G_od rho dv c/(1 - g rho dv) - off) scale, so
    dS/drho = scale G_od dv c / (1 - g rho dv)^2 and d|S_2|^2/drho = 2 Re(conj(S_2) dS_2/drho)."""
    s = fdfd64.sub_case([57])
    p = O.Problem.from_case(s)
    g, c, dv = s.G_dd[0, 0], s.c_d[0], s.dv[0]
    for rho in (0.0, 0.3, 1.0):
        den = 1.0 - g * rho * dv
        S = (s.c_o + s.G_od[:, 0] * rho * dv * c / den - s.s_off) * s.s_scale
        dS = s.s_scale * s.G_od[:, 0] * dv * c / den ** 2
        want = float(np.sum(s.obj_weights * 2.0 * np.real(np.conj(S) * dS)))
        got = O.objective_gradient(p, np.array([rho]))[0]
        assert abs(got - want) <= 1e-12 * abs(want)


def test_planted_gradient_mistakes_are_caught(fdfd64, monkeypatch):
    """Plausible slips in the gradient's chain rule fail the finite-difference pin."""
    p = O.Problem.from_case(fdfd64)
    rho = W.random_design(fdfd64.n_d, 4).astype(np.float64)
    ms = np.arange(0, 100, 9)
    fd = _grad_fd(p, rho, ms)
    real = O.pngf_oracle.port_projection
    plants = {
        "T without the V W term": lambda G, God, v: God.copy(),
        "transposed W in T": lambda G, God, v: God + (God * v[None, :]) @ O.maintained_inverse(G, v).T.conj(),
        "T scaled by V": lambda G, God, v: real(G, God, v) * v[None, :],
    }
    for what, bad in plants.items():
        monkeypatch.setattr(O.pngf_oracle, "port_projection", bad)
        g = O.objective_gradient(p, rho)
        assert np.max(np.abs(g[ms] - fd)) > 1e-3 * np.max(np.abs(fd)), what
    monkeypatch.undo()
    monkeypatch.setattr(O.pngf_oracle, "s_params", lambda o, off, sc: (o - off) * np.conj(sc))
    g = O.objective_gradient(p, rho)
    monkeypatch.undo()
    assert np.max(np.abs(g[ms] - fd)) > 1e-3 * np.max(np.abs(fd)), "conjugated scale"


# ---------------------------------------------------------------- tile flips on several systems
def test_combined_objective_rules():
    assert O.combined_objective([1.0, 3.0], O.OBJ_MAX_WEIGHTED_POWER, O.COMBINE_MEAN) == 2.0
    assert O.combined_objective([1.0, 3.0], O.OBJ_MAX_WEIGHTED_POWER, O.COMBINE_WORST) == 1.0
    assert O.combined_objective([1.0, 3.0], O.OBJ_MIN_INSERTION_LOSS, O.COMBINE_WORST) == 3.0


def test_single_pixel_tiles_reduce_to_pixel_dbs(fdfd64):
    """Tiles of one pixel on one system: the same trajectory as the pixel DBS
    (itself pinned by brute force above)."""
    p = O.Problem.from_case(fdfd64)
    b0 = W.random_design(fdfd64.n_d, 3)
    order = W.shuffled_order(fdfd64.n_d, 3, seed=2)
    ref = O.dbs(p, b0, order, tau=1e-9)
    tiles = np.arange(fdfd64.n_d, dtype=np.int32)[:, None]
    for combine in (O.COMBINE_MEAN, O.COMBINE_WORST):
        res = O.dbs_tiles([p], b0, tiles, order, tau=1e-9, combine=combine)
        assert [a[:3] for a in res.accepted] == [a[:3] for a in ref.accepted]
        assert res.f == ref.f and np.array_equal(res.b, ref.b)
    # two copies of one system under the mean: the same search again
    res2 = O.dbs_tiles([p, p], b0, tiles, order, tau=1e-9)
    assert [a[:3] for a in res2.accepted] == [a[:3] for a in ref.accepted]


@pytest.fixture(scope="module")
def tiny_two_freq(fdfd64):
    idx = [10 * x + y for x in range(3, 6) for y in range(3, 7)]  # 12 pixels, a 3 x 4 block
    l19 = W.get_case("fdfd64_l19")
    subs = [fdfd64.sub_case(idx), l19.sub_case(idx)]
    probs = [O.Problem.from_case(s) for s in subs]
    tables = [_enumerate(p) for p in probs]
    # pairs of vertically adjacent pixels of the block: 6 tiles of 2
    tiles = np.array([[4 * x + y, 4 * x + y + 1] for x in range(3) for y in (0, 2)], np.int32)
    return probs, tables, tiles


@pytest.mark.parametrize("combine", [O.COMBINE_MEAN, O.COMBINE_WORST])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tile_dbs_end_state_is_tile_locally_optimal(tiny_two_freq, combine, seed):
    probs, tables, tiles = tiny_two_freq
    kind = probs[0].obj_kind
    comb = np.array([O.combined_objective([t[m] for t in tables], kind, combine) for m in range(2 ** 12)])
    b0 = W.random_design(12, seed)
    order = np.tile(np.arange(len(tiles), dtype=np.int32), (30, 1))
    res = O.dbs_tiles(probs, b0, tiles, order, tau=1e-9, combine=combine)
    assert res.sweeps_done < 30
    assert res.f == comb[_code(res.b)]
    for tile in tiles:
        nb = O.flip_tile(res.b, tile)
        assert comb[_code(nb)] - res.f <= 1e-9 * abs(res.f)
    b, f = b0.copy(), comb[_code(b0)]
    for (_, _, ti, f_after) in res.accepted:
        b = O.flip_tile(b, tiles[ti])
        assert f_after == comb[_code(b)] and f_after > f + 1e-9 * abs(f)
        f = f_after
    # BEST takes the enumerated best tile neighbour every step
    best = O.dbs_tiles(probs, b0, tiles, order, tau=1e-9, mode=O.BEST_IMPROVEMENT, combine=combine)
    b = b0.copy()
    for (_, _, ti, f_after) in best.accepted:
        nbr = [comb[_code(O.flip_tile(b, t))] for t in tiles]
        assert ti == int(np.argmax(nbr))
        b = O.flip_tile(b, tiles[ti])
        assert f_after == comb[_code(b)]


def test_planted_tile_mistakes_are_caught(tiny_two_freq, monkeypatch):
    """Flipping only a tile's first pixel, or combining by the wrong rule, breaks
    the enumerated end-state pin."""
    probs, tables, tiles = tiny_two_freq
    kind = probs[0].obj_kind
    worst = np.array([O.combined_objective([t[m] for t in tables], kind, O.COMBINE_WORST) for m in range(2 ** 12)])
    order = np.tile(np.arange(len(tiles), dtype=np.int32), (30, 1))
    b0 = W.random_design(12, 1)
    real_flip = O.pngf_oracle.flip_tile
    monkeypatch.setattr(O.pngf_oracle, "flip_tile", lambda b, tile: real_flip(b, tile[:1]))
    res = O.dbs_tiles(probs, b0, tiles, order, tau=1e-9, combine=O.COMBINE_WORST)
    monkeypatch.undo()
    ok = all(worst[_code(real_flip(res.b, t))] - res.f <= 1e-9 * abs(res.f) for t in tiles)
    assert not (ok and res.f == worst[_code(res.b)]), "first pixel only"
    monkeypatch.setattr(O.pngf_oracle, "combined_objective", lambda fs, k, c: float(np.mean(fs)))
    res = O.dbs_tiles(probs, b0, tiles, order, tau=1e-9, combine=O.COMBINE_WORST)
    monkeypatch.undo()
    assert res.f != worst[_code(res.b)], "mean instead of min-max"


# ---------------------------------------------------------------- perfect-conductor (PEC) pixels, Eq. 2
def _full_structure_pec(case, b):
    """Port amplitudes of the full FDFD structure with every metal design node
    held at E = 0 (a perfect conductor), by a direct sparse solve without them."""
    import scipy.sparse.linalg as spl
    spec = W.SPECS[case.name]
    eps = W._eps_grid(spec)
    A, sxy = W.helmholtz_operator(eps, spec.npml, W._k(spec), npml_y=spec.npml_y)
    s, Pi = W._source_and_ports(spec, W._eps_grid(spec))
    metal = W._design_nodes(spec)[np.asarray(b, bool)]
    keep = np.setdiff1d(np.arange(A.shape[0]), metal)
    A = A.tocsr()
    E = np.zeros(A.shape[0], complex)
    E[keep] = spl.splu(A[keep][:, keep].tocsc()).solve(-(sxy * s)[keep])
    return E[W._design_nodes(spec)], Pi @ E


@pytest.mark.parametrize("name,seed", [("fdfd64", 3), ("fdfd128_metal", 2)])
def test_pec_system_equals_full_fdfd_with_conductors(name, seed, fdfd64, metal128):
    case = fdfd64 if name == "fdfd64" else metal128
    b = W.random_design(case.n_d, seed)
    ev = O.evaluate_pec(O.Problem.from_case(case), b)
    e_full, o_full = _full_structure_pec(case, b)
    assert np.max(np.abs(ev.o - o_full)) <= 1e-10 * np.max(np.abs(o_full))
    assert np.max(np.abs(ev.e - e_full)) <= 1e-10 * np.max(np.abs(e_full))
    assert np.max(np.abs(ev.e[b == 1])) <= 1e-12 * np.max(np.abs(e_full))  # no field inside the conductor


def test_pec_is_the_limit_of_lossy_metal(metal128):
    """The general-material system with eps_on = 1 + i s tends to the PEC system
    as s grows, the difference falling like 1/s."""
    p = O.Problem.from_case(metal128)
    b = W.random_design(metal128.n_d, 4)
    o_pec = O.evaluate_pec(p, b).o
    k2 = metal128.dv[0] / 1e4j  # k^2 of the workload (dv = k^2 * 1e4 i)
    errs = []
    for sig in (1e5, 1e7, 1e9):
        p.dv = np.full(metal128.n_d, k2 * sig * 1j)
        errs.append(np.max(np.abs(O.evaluate(p, b).o - o_pec)) / np.max(np.abs(o_pec)))
    assert errs[2] < 1e-6
    assert errs[1] < 3e-2 * errs[0] and errs[2] < 3e-2 * errs[1]


def test_pec_dbs_end_state_is_locally_optimal(fdfd64):
    s = _tiny(fdfd64)
    p = O.Problem.from_case(s)
    fs = np.array([O.evaluate_pec(p, np.array([(m >> i) & 1 for i in range(12)], np.uint8)).f
                   for m in range(2 ** 12)])
    for seed in (0, 1):
        res = O.dbs(p, W.random_design(12, seed), W.raster_order(12, 60), tau=1e-9, evaluator=O.evaluate_pec)
        assert res.sweeps_done < 60 and res.f == fs[_code(res.b)]
        for k in range(12):
            nb = res.b.copy(); nb[k] ^= 1
            assert fs[_code(nb)] - res.f <= 1e-9 * abs(res.f)


def test_planted_pec_mistakes_are_caught(metal128, monkeypatch):
    b = W.random_design(metal128.n_d, 2)
    _, o_full = _full_structure_pec(metal128, b)
    p = O.Problem.from_case(metal128)
    n = metal128.n_d
    plants = {
        "the paper's sign of G kept": lambda G, bb: np.eye(n) - np.diag(bb * 1.0) + np.diag(bb * 1.0) @ G,
        "(I - P) dropped": lambda G, bb: 1e-3 * np.eye(n) - np.diag(bb * 1.0) @ G,
        "G P instead of P G": lambda G, bb: np.eye(n) - np.diag(bb * 1.0) - G @ np.diag(bb * 1.0),
    }
    for what, bad in plants.items():
        monkeypatch.setattr(O.pngf_oracle, "pec_system", bad)
        o = O.evaluate_pec(p, b).o
        assert np.max(np.abs(o - o_full)) > 1e-6 * np.max(np.abs(o_full)), what
    monkeypatch.undo()
