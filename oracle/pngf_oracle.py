"""Plain, slow FP64 CPU oracle of the PNGF direct-binary-search hot path.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this module:
only the tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` call it.  It shares no code with the
CUDA path.

What it computes (notation of the field form; ``G`` is the design-to-design
numerical Green function, ``G_od`` the design-to-port functionals, ``c_d`` /
``c_o`` the incident fields, ``v = dv * b`` the per-pixel contrast of the
binary design ``b``):

* ``evaluate``: the objective of one design from scratch.  This is Eq. 7 of
  the paper (x_obj,n = G_obj C_n^-1 P_n e_inc + x_inc) in the generalised-
  material field form of Supplementary Note 4 (C = I + Y G and
  x_obj = G_obj C^-1 Y e_inc + x_inc, rewritten for the field e = G j):
  solve (I - G diag(v)) e = c_d with LAPACK zgesv (partial pivoting, FP64),
  then o = c_o + G_od (v * e).  The paper stresses that the low-rank path
  reaches exactly this value ("no approximations"), so the plain re-solve is
  the definition the fast path is checked against.
* ``dbs``: direct binary search as the paper's "Direct binary search
  optimization" section and Supplementary Fig. 1 describe it: from an initial
  design, visit tiles one at a time, flip, evaluate, keep the flip if the
  objective improved, otherwise undo it; stop when a whole pass over the tiles
  brings no improvement.  Every visited flip is re-solved from scratch.
* ``evaluate_pec``: the objective of a design of perfect-conductor pixels
  from the paper's own PEC system, Eq. 2: [(I - P) + P G] j = P e_inc (with
  this code's sign of G); ``dbs(..., evaluator=evaluate_pec)`` searches it.
* ``dbs_tiles``: DBS whose candidates flip a whole tile (several pixels at
  once, the paper's rank-M flips) on one or several systems that share the
  design (the paper's per-frequency systems), the per-system objectives
  combined into one by a mean or a min-max rule; every candidate re-solved.
* ``objective_gradient``: the gradient of the objective with respect to a
  continuous density of every pixel (Supplementary Note 5, field form).
* ``maintained_inverse`` / ``port_projection``: the plain definitions of the
  quantities a low-rank implementation keeps between iterations (the paper's
  C^-1, R = G_obj C^-1 and S = C^-1 P e_inc of Eqs. 11-12, in field form):
  W = M^-1 G and T = G_od (I + V W) with M = I - G V.

Readings where the paper is silent (all stated again in the project's design
notes): first-improvement in a caller-given visiting order (raster by
default); acceptance iff the gain exceeds tau * max(|f|, 1e-30); a candidate
whose solve is singular is rejected; S-parameters are the affine map
S_p = (o_p - s_off_p) * s_scale_p; objective kinds 0 (maximise
sum w_p |S_p|^2) and 1 (minimise sum w_p (1 - |S_p|)^2, the insertion-loss
objective of Supplementary Note 9).

Parity is pinned by the ``-m "not gpu"`` tests: a direct sparse solve of the
full modified FDFD structure, the one-pixel closed form, the zero-contrast
case, brute-force enumeration of every design on tiny regions, reciprocity
and energy conservation of lossless two-ports.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np
import scipy.linalg as sla

OBJ_MAX_WEIGHTED_POWER = 0
OBJ_MIN_INSERTION_LOSS = 1
FIRST_IMPROVEMENT = 0
BEST_IMPROVEMENT = 1
COMBINE_MEAN = 0   # arithmetic mean of the per-system objectives
COMBINE_WORST = 1  # min-max: the worst system (lowest maximised / highest minimised objective)


def system_matrix(G: np.ndarray, v: np.ndarray) -> np.ndarray:
    """M = I - G diag(v): the reduced field-form system (Supplementary Note 4)."""
    n = G.shape[0]
    return np.eye(n, dtype=np.complex128) - G * v[None, :]


def solve_field(G: np.ndarray, c_d: np.ndarray, v: np.ndarray) -> np.ndarray:
    """e = M^-1 c_d by LAPACK zgesv; raises numpy.linalg.LinAlgError if singular."""
    return sla.solve(system_matrix(G, v), c_d, check_finite=True)


def port_amplitudes(G_od: np.ndarray, c_o: np.ndarray, v: np.ndarray, e: np.ndarray) -> np.ndarray:
    """o = c_o + G_od (v * e): Eq. 5 with j = V e (polarisation currents)."""
    return c_o + G_od @ (v * e)


def s_params(o: np.ndarray, s_off: np.ndarray, s_scale: np.ndarray) -> np.ndarray:
    return (o - s_off) * s_scale


def objective(S: np.ndarray, kind: int, weights: np.ndarray) -> float:
    """Scalar figure of merit (Supplementary Note 9 style)."""
    a = np.abs(S)
    if kind == OBJ_MAX_WEIGHTED_POWER:
        return float(np.sum(weights * a * a))
    if kind == OBJ_MIN_INSERTION_LOSS:
        return float(np.sum(weights * (1.0 - a) ** 2))
    raise ValueError(f"unknown objective kind {kind}")


def improvement(f_new: float, f_old: float, kind: int) -> float:
    """Signed gain: positive means better."""
    return (f_new - f_old) if kind == OBJ_MAX_WEIGHTED_POWER else (f_old - f_new)


@dataclasses.dataclass
class Problem:
    """Arrays of one PNGF instance (complex128 unless noted)."""

    G: np.ndarray
    G_od: np.ndarray
    c_d: np.ndarray
    c_o: np.ndarray
    dv: np.ndarray
    s_off: np.ndarray
    s_scale: np.ndarray
    obj_kind: int
    obj_weights: np.ndarray

    @classmethod
    def from_case(cls, case) -> "Problem":
        return cls(case.G_dd, case.G_od, case.c_d, case.c_o, case.dv, case.s_off, case.s_scale,
                   int(case.obj_kind), np.asarray(case.obj_weights, dtype=np.float64))

    @property
    def n_d(self) -> int:
        return int(self.G.shape[0])


@dataclasses.dataclass
class Evaluation:
    e: np.ndarray
    o: np.ndarray
    S: np.ndarray
    f: float


def evaluate(p: Problem, b: np.ndarray) -> Evaluation:
    """Objective of design ``b`` from scratch (Eq. 7, field form)."""
    v = p.dv * np.asarray(b, dtype=np.float64)
    e = solve_field(p.G, p.c_d, v)
    o = port_amplitudes(p.G_od, p.c_o, v, e)
    S = s_params(o, p.s_off, p.s_scale)
    return Evaluation(e, o, S, objective(S, p.obj_kind, p.obj_weights))


def pec_system(G: np.ndarray, b: np.ndarray) -> np.ndarray:
    """C = (I - P) - P G: Eq. 2 of the paper, [(I - P) + P G] j = P e_inc, written
    with this code's sign of G (the total field is c_d + G j, the paper's is
    e_inc - G j), for a design of perfect electric conductor (PEC) pixels
    (P = diag(b), 1 = metal): on a metal pixel the total field vanishes, on an
    empty pixel the current does."""
    n = G.shape[0]
    p = np.asarray(b, dtype=np.float64)
    return np.eye(n, dtype=np.complex128) - np.diag(p) - p[:, None] * G  # P G: rows of G scaled by P


def evaluate_pec(p: Problem, b: np.ndarray) -> Evaluation:
    """Objective of a PEC design from scratch: C j = P c_d (Eq. 2), o = c_o + G_od j
    (Eq. 5); ``e`` is the total field c_d + G j (zero on metal)."""
    b = np.asarray(b, dtype=np.uint8)
    j = sla.solve(pec_system(p.G, b), b * p.c_d, check_finite=True)
    o = p.c_o + p.G_od @ j
    S = s_params(o, p.s_off, p.s_scale)
    # e = c_d + G j, summed by numpy itself (a threaded BLAS matrix-vector
    # product of this size spends far longer starting threads than computing)
    return Evaluation(p.c_d + np.einsum("ij,j->i", p.G, j), o, S, objective(S, p.obj_kind, p.obj_weights))


def candidate_objectives(p: Problem, b: np.ndarray, pixels, evaluator=None) -> np.ndarray:
    """Objective after flipping each listed pixel alone (re-solved from scratch).

    A singular candidate gets NaN.  ``evaluator``: evaluate (default) or evaluate_pec.
    """
    ev_fn = evaluate if evaluator is None else evaluator
    out = np.empty(len(pixels), dtype=np.float64)
    b = np.asarray(b, dtype=np.uint8)
    for i, k in enumerate(pixels):
        b2 = b.copy()
        b2[k] ^= 1
        try:
            out[i] = ev_fn(p, b2).f
        except np.linalg.LinAlgError:
            out[i] = np.nan
    return out


def candidate_ports(p: Problem, b: np.ndarray, pixels) -> np.ndarray:
    """Port amplitudes after flipping each listed pixel alone, (len, n_o)."""
    b = np.asarray(b, dtype=np.uint8)
    out = np.empty((len(pixels), p.G_od.shape[0]), dtype=np.complex128)
    for i, k in enumerate(pixels):
        b2 = b.copy()
        b2[k] ^= 1
        out[i] = evaluate(p, b2).o
    return out


def maintained_inverse(G: np.ndarray, v: np.ndarray) -> np.ndarray:
    """W = M^-1 G (the inverse the paper maintains, in field form)."""
    return sla.solve(system_matrix(G, v), G)


def port_projection(G: np.ndarray, G_od: np.ndarray, v: np.ndarray) -> np.ndarray:
    """T = G_od (I + V W): port response to a unit change of a pixel's current."""
    W = maintained_inverse(G, v)
    return G_od + (G_od * v[None, :]) @ W


def objective_gradient(p: Problem, rho: np.ndarray) -> np.ndarray:
    """df/drho_m of the objective for the density parameterisation v = dv * rho.

    Supplementary Note 5 gives the gradient of a real objective with respect
    to the design parameters through the chain rule with Wirtinger
    derivatives, grad f = 2 Re[(df/dx_obj)(dx_obj/dy)(dy/dp)], where the
    derivative of x_obj with respect to one design entry is the m-th column of
    R = G_obj C^-1 times the m-th entry of (e_inc - S) (its elementwise
    form, O(N_obj) work per entry).  In the field form used here
    (x_obj = o = c_o + G_od V e, M = I - G V, M e = c_d) the same product rule
    gives do/dv_m = T[:, m] e_m with T = G_od (I + V W), W = M^-1 G; the design
    parameter is the real density rho_m of pixel m (v_m = rho_m dv_m, so
    dv_m/drho_m = dv_m; rho in {0, 1} is the binary design).  The objective
    is f = sum_p phi_p(S_p), S_p = (o_p - off_p) scale_p, with Wirtinger
    derivatives dphi/dS = w conj(S) for w |S|^2 and
    -w (1 - |S|) conj(S) / |S| for w (1 - |S|)^2 (0 where S = 0, a cusp).
    """
    rho = np.asarray(rho, dtype=np.float64)
    v = p.dv * rho
    e = solve_field(p.G, p.c_d, v)
    o = port_amplitudes(p.G_od, p.c_o, v, e)
    S = s_params(o, p.s_off, p.s_scale)
    if p.obj_kind == OBJ_MAX_WEIGHTED_POWER:
        dfdS = p.obj_weights * np.conj(S)
    elif p.obj_kind == OBJ_MIN_INSERTION_LOSS:
        a = np.abs(S)
        dfdS = np.where(a > 0, -p.obj_weights * (1.0 - a) * np.conj(S) / np.where(a > 0, a, 1.0), 0.0)
    else:
        raise ValueError(f"unknown objective kind {p.obj_kind}")
    T = port_projection(p.G, p.G_od, v)
    dodrho = T * (e * p.dv)[None, :]  # (n_o, n_d): do_p / drho_m
    return 2.0 * np.real((dfdS * p.s_scale) @ dodrho)


@dataclasses.dataclass
class DbsResult:
    accepted: List[tuple]  # (sweep, position, pixel, f_after)
    b: np.ndarray
    f: float
    o: np.ndarray
    S: np.ndarray
    n_evals: int
    sweeps_done: int
    min_abs_margin: float  # smallest |gain - tau*max(|f|,1e-30)| over all decisions
    margins: Optional[list] = None  # FIRST mode: (sweep, position, margin, f before) per decision


def dbs(p: Problem, b0: np.ndarray, order: np.ndarray, tau: float = 1e-9,
        mode: int = FIRST_IMPROVEMENT, max_evals: Optional[int] = None,
        keep_margins: bool = False, evaluator=None) -> DbsResult:
    """Direct binary search, every candidate re-solved from scratch.

    ``order`` has shape (n_sweeps, n_d): the visiting order of each sweep.
    FIRST: visit positions in order; keep the first flip that improves.
    BEST: at each step flip the best improving pixel of the whole region
    (ties -> lowest pixel index) and count one sweep per step.
    A sweep without any accepted flip ends the search (converged).
    ``max_evals`` bounds the work (used for timing samples).  ``evaluator``:
    evaluate (default, the general-material field form) or evaluate_pec.
    """
    evaluate_ = evaluate if evaluator is None else evaluator
    b = np.asarray(b0, dtype=np.uint8).copy()
    cur = evaluate_(p, b)
    f = cur.f
    accepted: List[tuple] = []
    n_evals = 0
    min_margin = np.inf
    margins = [] if keep_margins else None
    sweeps_done = 0
    order = np.atleast_2d(np.asarray(order))
    for s in range(order.shape[0]):
        any_accept = False
        if mode == FIRST_IMPROVEMENT:
            for t, k in enumerate(order[s]):
                if max_evals is not None and n_evals >= max_evals:
                    break
                b2 = b.copy()
                b2[k] ^= 1
                n_evals += 1
                try:
                    ev = evaluate_(p, b2)
                except np.linalg.LinAlgError:
                    continue
                margin = improvement(ev.f, f, p.obj_kind) - tau * max(abs(f), 1e-30)
                min_margin = min(min_margin, abs(margin))
                if keep_margins:
                    margins.append((s, t, margin, f))
                if margin > 0:
                    b, f, cur = b2, ev.f, ev
                    accepted.append((s, t, int(k), f))
                    any_accept = True
        else:
            cand = np.arange(p.n_d)
            fs = candidate_objectives(p, b, cand, evaluator)
            n_evals += p.n_d
            gains = np.array([improvement(x, f, p.obj_kind) if np.isfinite(x) else -np.inf for x in fs])
            m = gains - tau * max(abs(f), 1e-30)
            min_margin = min(min_margin, float(np.min(np.abs(m[np.isfinite(m)]))))
            best = int(np.argmax(gains))  # argmax returns the lowest index among ties
            if m[best] > 0:
                b = b.copy()
                b[best] ^= 1
                cur = evaluate_(p, b)
                f = cur.f
                accepted.append((s, 0, best, f))
                any_accept = True
        sweeps_done += 1
        if not any_accept or (max_evals is not None and n_evals >= max_evals):
            break
    return DbsResult(accepted, b, f, cur.o, cur.S, n_evals, sweeps_done, float(min_margin), margins)


# ---------------------------------------------------------------- tile flips and several systems
def combined_objective(fs, kind: int, combine: int) -> float:
    """One scalar from the objectives of several systems (Supplementary Note 9:
    the per-frequency objectives are combined by a mean or a min-max rule)."""
    fs = np.asarray(fs, dtype=np.float64)
    if combine == COMBINE_MEAN:
        return float(np.mean(fs))
    if combine == COMBINE_WORST:
        return float(np.min(fs)) if kind == OBJ_MAX_WEIGHTED_POWER else float(np.max(fs))
    raise ValueError(f"unknown combine rule {combine}")


def flip_tile(b: np.ndarray, tile) -> np.ndarray:
    """The design with every pixel of one tile flipped (negative entries pad a tile)."""
    b2 = np.asarray(b, dtype=np.uint8).copy()
    for k in tile:
        if k >= 0:
            b2[k] ^= 1
    return b2


def tile_candidate_objectives(problems, b, tiles, combine: int) -> np.ndarray:
    """Combined objective after flipping each tile alone, re-solved from scratch
    in every system; a candidate singular in any system gets NaN."""
    out = np.empty(len(tiles), dtype=np.float64)
    for i, tile in enumerate(tiles):
        b2 = flip_tile(b, tile)
        try:
            out[i] = combined_objective([evaluate(p, b2).f for p in problems], problems[0].obj_kind, combine)
        except np.linalg.LinAlgError:
            out[i] = np.nan
    return out


def dbs_tiles(problems, b0: np.ndarray, tiles, order: np.ndarray, tau: float = 1e-9,
              mode: int = FIRST_IMPROVEMENT, combine: int = COMBINE_MEAN) -> DbsResult:
    """Direct binary search over tile flips on one or several systems sharing the design.

    The paper's DBS flips a tile -- the M unknowns of a block of cells, and in
    its designs 2 to 4 symmetry-tied tiles at once ("Low-rank update
    evaluation"; Methods, "Optimization parameters") -- and its multi-frequency
    designs evaluate one system per frequency on the same design ("Computational
    efficiency") with the per-frequency objectives combined into one scalar
    (Supplementary Note 9).  Here every candidate flips all pixels of one tile
    (a row of ``tiles``; negative entries pad), every system is re-solved from
    scratch, and the combined objective decides: FIRST keeps the first
    improving tile of the visiting order (rows of ``order`` are permutations of
    the tile indices), BEST the best improving tile (ties -> lowest tile index).
    ``trace`` entries are (sweep, position, tile, combined objective after).
    """
    kind = problems[0].obj_kind
    b = np.asarray(b0, dtype=np.uint8).copy()

    def fcomb(bb):
        evs = [evaluate(p, bb) for p in problems]
        return combined_objective([ev.f for ev in evs], kind, combine), evs

    f, evs = fcomb(b)
    accepted: List[tuple] = []
    n_evals, sweeps_done, min_margin = 0, 0, np.inf
    order = np.atleast_2d(np.asarray(order))
    n_t = len(tiles)
    for s in range(order.shape[0]):
        any_accept = False
        if mode == FIRST_IMPROVEMENT:
            for t, ti in enumerate(order[s]):
                b2 = flip_tile(b, tiles[ti])
                n_evals += 1
                try:
                    f2, evs2 = fcomb(b2)
                except np.linalg.LinAlgError:
                    continue
                margin = improvement(f2, f, kind) - tau * max(abs(f), 1e-30)
                min_margin = min(min_margin, abs(margin))
                if margin > 0:
                    b, f, evs = b2, f2, evs2
                    accepted.append((s, t, int(ti), f))
                    any_accept = True
        else:
            fs = tile_candidate_objectives(problems, b, tiles, combine)
            n_evals += n_t
            gains = np.array([improvement(x, f, kind) if np.isfinite(x) else -np.inf for x in fs])
            m = gains - tau * max(abs(f), 1e-30)
            min_margin = min(min_margin, float(np.min(np.abs(m[np.isfinite(m)]))))
            best = int(np.argmax(gains))
            if m[best] > 0:
                b = flip_tile(b, tiles[best])
                f, evs = fcomb(b)
                accepted.append((s, 0, best, f))
                any_accept = True
        sweeps_done += 1
        if not any_accept:
            break
    res = DbsResult(accepted, b, f, evs[0].o, evs[0].S, n_evals, sweeps_done, float(min_margin))
    res.o_all = [ev.o for ev in evs]
    return res
