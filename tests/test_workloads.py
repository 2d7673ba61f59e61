"""Input-generator invariants (CPU): the precomputed G and its physics.

These pin the synthetic stand-ins for the paper's precomputed Green functions
(section "Precomputation", Eq. 3) to physics that does not depend on the code
under test: symmetry of the reciprocal operator, reciprocity of independent
full solves, PML absorption, energy conservation of a lossless two-port and
the closed-form 2D Green function.
"""
import numpy as np
import pytest
import scipy.integrate as si
import scipy.linalg as sla
import scipy.sparse.linalg as spl
from scipy.special import hankel1

from paper_2501_18054_gb300 import workloads as W
import oracle as O


def test_operator_is_complex_symmetric():
    eps = W._eps_grid(W.SPECS["fdfd128_metal"])
    A, _ = W.helmholtz_operator(eps, 12)
    D = (A - A.T).tocoo()
    assert D.nnz == 0 or np.max(np.abs(D.data)) == 0.0


def test_reciprocity_of_full_solves():
    """Field at a due to a point source at b equals field at b due to a source at a."""
    spec = W.SPECS["fdfd128_metal"]
    eps = W._eps_grid(spec)
    A, sxy = W.helmholtz_operator(eps, spec.npml)
    lu = spl.splu(A.tocsc())
    n = spec.n
    a, b = 40 * n + 61, 90 * n + 75  # one in the slab, one in air
    sa = np.zeros(n * n, complex); sa[a] = 1.0
    sb = np.zeros(n * n, complex); sb[b] = 1.0
    Ea = lu.solve(-sa * sxy)
    Eb = lu.solve(-sb * sxy)
    assert abs(Ea[b] - Eb[a]) <= 1e-12 * abs(Ea[b])


def test_generated_G_is_symmetric_before_symmetrisation():
    """The Schur-complement inverse is symmetric to rounding; the stored G exactly."""
    c = W.make_fdfd_case("fdfd64", cache=False)
    assert np.array_equal(c.G_dd, c.G_dd.T)
    # recompute without the final symmetrisation through an independent path:
    # columns of -A^-1 B by full sparse solves
    spec = W.SPECS["fdfd64"]
    eps = W._eps_grid(spec)
    A, _ = W.helmholtz_operator(eps, spec.npml)
    d = W._design_nodes(spec)
    rhs = np.zeros((A.shape[0], 7), complex)
    cols = [0, 13, 27, 50, 64, 88, 99]
    rhs[d[cols], np.arange(7)] = 1.0
    X = spl.splu(A.tocsc()).solve(rhs)
    G_cols = -X[d, :]
    assert np.max(np.abs(G_cols - c.G_dd[:, cols])) <= 1e-12 * np.max(np.abs(c.G_dd))


def test_pml_absorbs():
    """A point source in a small PML box matches the same source in a 3x larger box."""
    k = W.K_CELL
    small, big, npml = 64, 192, 10
    eps_s = np.ones((small, small), complex)
    eps_b = np.ones((big, big), complex)
    As, sxs = W.helmholtz_operator(eps_s, npml)
    Ab, sxb = W.helmholtz_operator(eps_b, npml)
    src_s = np.zeros((small, small), complex); src_s[32, 32] = 1.0
    src_b = np.zeros((big, big), complex); src_b[96, 96] = 1.0
    Es = spl.splu(As.tocsc()).solve(-sxs * src_s.ravel()).reshape(small, small)
    Eb = spl.splu(Ab.tocsc()).solve(-sxb * src_b.ravel()).reshape(big, big)
    inner_s = Es[npml + 2:small - npml - 2, npml + 2:small - npml - 2]
    o = 96 - 32
    inner_b = Eb[o + npml + 2:o + small - npml - 2, o + npml + 2:o + small - npml - 2]
    err = np.max(np.abs(inner_s - inner_b)) / np.max(np.abs(inner_b))
    assert err < 2e-3, err
    # and the discrete field approaches the continuum Green function (i/4) H0(k r)
    r = np.array([6.0, 8.0, 10.0])
    g = 0.25j * hankel1(0, k * r)
    num = Eb[96 + r.astype(int), 96]  # A E = -delta:  E = -A^-1 delta = G delta ~ g
    assert np.max(np.abs(num - g) / np.abs(g)) < 0.05


def _two_port_spec():
    # closed parallel-plate guide: Dirichlet walls along y (18 interior nodes),
    # PML along x; only the first guided mode propagates at eps = 1
    return W.FdfdSpec("pp_two_port", 220, 30, 1.0, (100, 0, 20, 18), 1.0, 4.0, slab=None,
                      source="mode", source_x=40, ports_x=(60, 61, 170, 171), port_kind="mode",
                      norm="incident", ny=18, npml_y=0, obj_weights=(0.0, 0.0, 1.0, 0.0))


def _two_line(a0, a1, beta):
    """Forward / backward amplitudes from the modal amplitude on two adjacent lines."""
    M = np.array([[1.0, 1.0], [np.exp(1j * beta), np.exp(-1j * beta)]])
    return np.linalg.solve(M, np.array([a0, a1]))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_lossless_two_port_conserves_energy(seed):
    """|S11|^2 + |S21|^2 = 1 through the reduced system (oracle) on a lossless guide."""
    spec = _two_port_spec()
    case = W.make_fdfd_case(spec, cache=False)
    p = O.Problem.from_case(case)
    ny = spec.ny
    kyd2 = 2.0 * (1.0 - np.cos(np.pi / (ny + 1)))
    k = W.K_CELL
    beta = np.arccos(1.0 - (k * k - kyd2) / 2.0)  # 2(cos b - 1) + k^2 - ky^2 = 0
    b = W.random_design(case.n_d, seed)
    o = O.evaluate(p, b).o
    inc = case.c_o  # empty design: only the forward wave
    A1, _ = _two_line(inc[0], inc[1], beta)
    F1, B1 = _two_line(o[0], o[1], beta)
    F2, B2 = _two_line(o[2], o[3], beta)
    # the incident wave is unchanged by the design (up to evanescent tails of higher modes)
    assert abs(F1 - A1) < 1e-6 * abs(A1)
    S11 = B1 / A1
    S21 = F2 / A1
    assert abs(B2) < 1e-4 * abs(A1)  # nothing comes back from the right PML
    assert abs(abs(S11) ** 2 + abs(S21) ** 2 - 1.0) < 1e-4
    assert abs(S11) > 1e-3  # the design actually scatters
    # the oracle's S-parameters (the recipe's affine map of the reduced-system
    # ports) are these modal values: port 1's line reports the reflected wave,
    # port 2's line the transmitted one relative to the empty guide's
    S = O.evaluate(p, b).S
    F2e, _ = _two_line(inc[2], inc[3], beta)
    assert abs(S[0] - S11) < 2e-6
    assert abs(S[2] - F2 / F2e) < 1e-6
    assert abs(abs(S[0]) ** 2 + abs(S[2]) ** 2 - 1.0) < 1e-4


def test_hankel_self_term_matches_quadrature():
    k = W.K_CELL
    a = 1.0 / np.sqrt(np.pi)
    re = si.quad(lambda r: 2 * np.pi * r * np.real(0.25j * hankel1(0, k * r)), 0, a, limit=200)[0]
    im = si.quad(lambda r: 2 * np.pi * r * np.imag(0.25j * hankel1(0, k * r)), 0, a, limit=200)[0]
    val = W.hankel_self_term(k)
    assert abs(val - (re + 1j * im)) < 1e-9 * abs(val)


def test_hankel_case_structure():
    c = W.make_hankel_case(side=12, cache=False)
    assert c.n_d == 144 and c.n_o == 4
    assert np.array_equal(c.G_dd, c.G_dd.T)
    k = W.K_CELL
    i, j = 5, 5 + 3 * 12 + 4  # offset (3, 4) -> r = 5
    assert abs(c.G_dd[i, j] - 0.25j * hankel1(0, 5 * k)) < 1e-14
    # port points sit at cell corners, never on a pixel centre
    pts = np.asarray(c.meta["ports"])
    assert np.all(np.abs(pts - np.round(pts)) == 0.5)


def test_sub_case_is_principal_block():
    c = W.make_fdfd_case("fdfd64", cache=False)
    idx = np.array([3, 7, 40, 41, 99])
    s = c.sub_case(idx)
    assert np.array_equal(s.G_dd, c.G_dd[np.ix_(idx, idx)])
    assert np.array_equal(s.G_od, c.G_od[:, idx])


def test_seeded_designs_and_orders():
    b1 = W.random_design(100, 5)
    assert np.array_equal(b1, W.random_design(100, 5))
    assert 30 < b1.sum() < 70
    o = W.shuffled_order(50, 3, 7)
    assert o.shape == (3, 50)
    for row in o:
        assert np.array_equal(np.sort(row), np.arange(50))
    assert not np.array_equal(o[0], o[1])
