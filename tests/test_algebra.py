"""The low-rank algebra the CUDA path implements, against the oracle's plain
re-solves (CPU only).

Field-form restatement of the paper's Woodbury identity (Eq. 9) for a rank-1
change (Sherman-Morrison) and of the candidate evaluation through the kept
quantities R, S, x_obj (Eqs. 11-14), written out here in numpy independently
of both the oracle and the kernels:

  d_k = 1 - delta W_kk,  alpha = delta / d_k,  o^(k) = o + alpha e_k T[:,k]
  keep:  W += alpha c c^T, T += alpha T[:,k] c^T, e += alpha e_k c,  c = W[:,k]
  refresh: e += r + W V r (r = c_d - M e), T += R + R V W (R = G_od - T M^T)
"""
import numpy as np
import pytest

from paper_2501_18054_gb300 import workloads as W
import oracle as O


def _random_symmetric_problem(n=40, n_o=3, seed=0):
    rng = np.random.default_rng(seed)
    A = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    G = 0.5 * (A + A.T) + 0.3 * np.eye(n)
    God = rng.standard_normal((n_o, n)) + 1j * rng.standard_normal((n_o, n))
    cd = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    co = rng.standard_normal(n_o) + 1j * rng.standard_normal(n_o)
    dv = (0.5 + 0.4j) * np.ones(n)
    return O.Problem(G, God, cd, co, dv, np.zeros(n_o, complex), np.ones(n_o, complex),
                     O.OBJ_MAX_WEIGHTED_POWER, np.ones(n_o))


def _state(p, b):
    v = p.dv * b
    Wm = O.maintained_inverse(p.G, v)
    T = O.port_projection(p.G, p.G_od, v)
    ev = O.evaluate(p, b)
    return Wm, T, ev.e, ev.o


@pytest.mark.parametrize("seed", [0, 1])
def test_candidate_ports_match_resolve(seed):
    p = _random_symmetric_problem(seed=seed)
    b = (np.random.default_rng(seed).random(p.n_d) < 0.5).astype(np.uint8)
    Wm, T, e, o = _state(p, b)
    cand = np.arange(p.n_d)
    ref = O.candidate_ports(p, b, cand)
    delta = np.where(b == 0, p.dv, -p.dv)
    d = 1.0 - delta * np.diag(Wm)
    alpha = delta / d
    fast = o[None, :] + (alpha * e)[:, None] * T.T
    assert np.max(np.abs(fast - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("seed", [0, 1])
def test_kept_flip_update_matches_resolve(seed):
    p = _random_symmetric_problem(seed=seed)
    rng = np.random.default_rng(10 + seed)
    b = (rng.random(p.n_d) < 0.5).astype(np.uint8)
    Wm, T, e, o = _state(p, b)
    for k in rng.permutation(p.n_d)[:6]:
        delta = -p.dv[k] if b[k] else p.dv[k]
        d = 1.0 - delta * Wm[k, k]
        alpha = delta / d
        c = Wm[:, k].copy()
        ek, Tk = e[k], T[:, k].copy()
        Wm = Wm + alpha * np.outer(c, c)
        T = T + alpha * np.outer(Tk, c)
        e = e + alpha * ek * c
        o = o + alpha * ek * Tk
        b[k] ^= 1
        W2, T2, e2, o2 = _state(p, b)
        assert np.max(np.abs(Wm - W2)) < 1e-11 * np.max(np.abs(W2))
        assert np.max(np.abs(T - T2)) < 1e-11 * np.max(np.abs(T2))
        assert np.max(np.abs(e - e2)) < 1e-11 * np.max(np.abs(e2))
        assert np.max(np.abs(o - o2)) < 1e-11 * np.max(np.abs(o2))


def test_identities():
    p = _random_symmetric_problem(seed=3)
    b = (np.random.default_rng(3).random(p.n_d) < 0.5).astype(np.uint8)
    v = p.dv * b
    M = O.system_matrix(p.G, v)
    Wm = O.maintained_inverse(p.G, v)
    Minv = np.linalg.inv(M)
    assert np.max(np.abs(Minv - (np.eye(p.n_d) + Wm * v[None, :]))) < 1e-12
    e = O.evaluate(p, b).e
    for k in np.flatnonzero(b)[:4]:  # turn-off flips: d_k = (M^-1)_kk
        delta = -p.dv[k]
        d = 1.0 - delta * Wm[k, k]
        assert abs(d - Minv[k, k]) < 1e-12
        b2 = b.copy(); b2[k] = 0
        e2 = O.evaluate(p, b2).e
        assert abs(e2[k] - e[k] / d) < 1e-12 * abs(e2[k])


def test_refresh_step_restores_accuracy():
    """One refinement step with a perturbed W brings e and T back to the re-solve."""
    case = W.make_fdfd_case("fdfd64")
    p = O.Problem.from_case(case)
    b = W.random_design(case.n_d, 2)
    v = p.dv * b
    Wm, T, e, o = _state(p, b)
    rng = np.random.default_rng(0)
    Wp = Wm * (1 + 1e-7 * rng.standard_normal(Wm.shape))  # inverse known to 1e-7
    e_bad = e * (1 + 1e-6 * rng.standard_normal(e.shape))
    T_bad = T * (1 + 1e-6 * rng.standard_normal(T.shape))
    r = p.c_d - (e_bad - p.G @ (v * e_bad))
    e_new = e_bad + r + Wp @ (v * r)
    R = p.G_od - (T_bad - (T_bad * v[None, :]) @ p.G)
    T_new = T_bad + R + (R * v[None, :]) @ Wp
    assert np.max(np.abs(e_new - e)) < 1e-11 * np.max(np.abs(e))
    assert np.max(np.abs(T_new - T)) < 1e-11 * np.max(np.abs(T))
    o_new = p.c_o + p.G_od @ (v * e_new)
    assert np.max(np.abs(o_new - o)) < 1e-11 * np.max(np.abs(o))
