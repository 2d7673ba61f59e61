"""Seeded synthetic PNGF workloads (static-structure precompute = input generation).

This module builds the inputs of the direct-binary-search (DBS) hot path: the
design-to-design numerical Green function ``G_dd``, the design-to-port
functionals ``G_od``, the incident fields ``c_d`` / ``c_o`` on the design pixels
and at the ports, the per-pixel contrast ``dv`` and the S-parameter
normalisation.  It holds none of the DBS / low-rank-update arithmetic: it is the
precompute stage the paper treats as a one-off cost ("Precomputation", Eq. 3
``G = B^T A^-1 B`` and the objective functional ``G_obj = W^T A^-1 B`` of
Eq. 5), done here for a 2D TM scalar FDFD operator (Supplementary Note 2 reduced
to the E_z polarisation).  It is shared, unchanged, by the oracle tests and the
CUDA path.

Conventions (time dependence exp(-i w t), lengths in grid cells, k = k0*dx):

* background operator  A_bg = L_pml + k^2 diag(eps_bg * s_x s_y)  (symmetrised
  stretched-coordinate PML, so A_bg = A_bg^T),
* total field          A E = -S  with  A = A_bg + k^2 B diag(d_eps) B^T,
* reduced system       (I - G V) e = c_d,  G = -B^T A_bg^-1 B,  V = diag(v),
                       v_k = k^2 * d_eps_k * b_k,
* port amplitudes      o = c_o + G_od V e,  G_od = -Pi^T A_bg^-1 B,
* S-parameters         S_p = (o_p - s_off_p) * s_scale_p.

``G`` is obtained from the Schur complement of ``A_bg`` on the design block
(the reduction that the augmented partial factorisation of the paper's
Precomputation section performs): with d = design nodes and r = the rest,
(A_bg^-1)_dd = (A_dd - A_dr A_rr^-1 A_rd)^-1, and ``A_rd`` is non-zero only on
the design boundary, so only a perimeter's worth of sparse solves is needed.
"""
from __future__ import annotations

import dataclasses
import hashlib
import json
import os
import tempfile
from typing import Optional, Sequence

import numpy as np

OBJ_MAX_WEIGHTED_POWER = 0  # f = sum_p w_p |S_p|^2, maximised
OBJ_MIN_INSERTION_LOSS = 1  # f = sum_p w_p (1 - |S_p|)^2, minimised

LAMBDA_CELLS = 20.0  # dx = lambda / 20 in every workload
RECIPE_VERSION = "2"  # part of every cache key: bump when a generated array changes
K_CELL = 2.0 * np.pi / LAMBDA_CELLS  # k0 * dx


@dataclasses.dataclass
class Case:
    """One PNGF problem instance (all complex arrays are complex128)."""

    name: str
    G_dd: np.ndarray  # (n_d, n_d), complex symmetric
    G_od: np.ndarray  # (n_o, n_d)
    c_d: np.ndarray  # (n_d,)
    c_o: np.ndarray  # (n_o,)
    dv: np.ndarray  # (n_d,) v_k for an "on" pixel: k^2 * (eps_on - eps_off)
    s_off: np.ndarray  # (n_o,)
    s_scale: np.ndarray  # (n_o,)
    obj_kind: int
    obj_weights: np.ndarray  # (n_o,) float64
    meta: dict

    @property
    def n_d(self) -> int:
        return int(self.G_dd.shape[0])

    @property
    def n_o(self) -> int:
        return int(self.G_od.shape[0])

    def sub_case(self, idx: Sequence[int], name: Optional[str] = None) -> "Case":
        """Principal sub-block: pixels outside ``idx`` stay at the background.

        Exact, because the reduced Green function of a subset of pixels is the
        principal sub-block of the larger one (B_s^T A^-1 B_s).
        """
        idx = np.asarray(idx, dtype=np.int64)
        return Case(
            name=name or f"{self.name}[sub{len(idx)}]",
            G_dd=np.ascontiguousarray(self.G_dd[np.ix_(idx, idx)]),
            G_od=np.ascontiguousarray(self.G_od[:, idx]),
            c_d=np.ascontiguousarray(self.c_d[idx]),
            c_o=self.c_o.copy(),
            dv=np.ascontiguousarray(self.dv[idx]),
            s_off=self.s_off.copy(),
            s_scale=self.s_scale.copy(),
            obj_kind=self.obj_kind,
            obj_weights=self.obj_weights.copy(),
            meta=dict(self.meta, parent=self.name, sub_pixels=len(idx)),
        )


# ----------------------------------------------------------------------------
# 2D TM FDFD with a symmetrised stretched-coordinate PML
# ----------------------------------------------------------------------------

def pml_stretch(n: int, npml: int, k: float, r0: float = 1e-8, m: int = 3):
    """Stretch factors at integer nodes (n,) and at half nodes i-1/2, i = 0..n (n+1,).

    s(rho) = 1 + i*sigma_max*(rho/npml)^m, rho = depth into the layer in cells;
    sigma_max is chosen so that a normally incident wave comes back with
    amplitude r0 after the round trip through the layer.
    """
    sigma_max = -(m + 1) * np.log(r0) / (2.0 * k * npml) if npml > 0 else 0.0
    lo, hi = float(npml), float(n - 1 - npml)

    def s_of(x):
        rho = np.maximum(np.maximum(lo - x, x - hi), 0.0)
        return 1.0 + 1j * sigma_max * (rho / max(npml, 1)) ** m

    xi = np.arange(n, dtype=np.float64)
    return s_of(xi), s_of(np.arange(n + 1, dtype=np.float64) - 0.5)


def helmholtz_operator(eps: np.ndarray, npml: int, k: float = K_CELL, npml_y: Optional[int] = None):
    """Sparse symmetric A = L_pml + k^2 diag(eps s_x s_y) on an (nx, ny) grid.

    ``npml_y`` (default ``npml``) sets the layer along y; 0 leaves plain
    Dirichlet walls there (a closed parallel-plate guide).

    Node (ix, iy) has flat index ix*ny + iy; the field vanishes outside the
    grid (Dirichlet ghost nodes).  The x-coupling of nodes i and i+1 is
    s_y / s_x(i+1/2), the y-coupling s_x / s_y(j+1/2): the stretched-coordinate
    operator multiplied through by s_x s_y, which keeps it complex symmetric.
    Returns (A (csc), sxy) where sxy = s_x s_y per node (the source scaling).
    """
    import scipy.sparse as sp

    nx, ny = eps.shape
    sx, sxh = pml_stretch(nx, npml, k)
    sy, syh = pml_stretch(ny, npml if npml_y is None else npml_y, k)
    idx = np.arange(nx * ny).reshape(nx, ny)
    cxf = sy[None, :] / sxh[:, None]  # (nx+1, ny): coupling across half node i-1/2
    cyf = sx[:, None] / syh[None, :]  # (nx, ny+1)
    diag = (k * k) * eps.astype(np.complex128) * sx[:, None] * sy[None, :]
    diag -= cxf[:-1, :] + cxf[1:, :] + cyf[:, :-1] + cyf[:, 1:]
    cx = cxf[1:-1, :]  # interior x-links (nx-1, ny)
    cy = cyf[:, 1:-1]  # interior y-links (nx, ny-1)
    ax, bx = idx[:-1, :].ravel(), idx[1:, :].ravel()
    ay, by = idx[:, :-1].ravel(), idx[:, 1:].ravel()
    rows = np.concatenate([ax, bx, ay, by, idx.ravel()])
    cols = np.concatenate([bx, ax, by, ay, idx.ravel()])
    vals = np.concatenate([cx.ravel(), cx.ravel(), cy.ravel(), cy.ravel(), diag.ravel()])
    A = sp.csc_matrix((vals, (rows, cols)), shape=(nx * ny, nx * ny))
    return A, (sx[:, None] * sy[None, :]).ravel()


def slab_mode(eps_col: np.ndarray, k: float = K_CELL):
    """Fundamental guided mode of a 1D transverse cross-section.

    Discrete eigenproblem (D_yy + k^2 eps(y)) phi = beta^2 phi with Dirichlet
    ends; returns (phi normalised to sum phi^2 = 1 with a positive peak, beta).
    """
    import scipy.linalg as sla

    n = len(eps_col)
    d = -2.0 * np.ones(n) + k * k * np.real(eps_col)
    w, v = sla.eigh_tridiagonal(d, np.ones(n - 1))
    j = int(np.argmax(w))
    phi = v[:, j]
    phi = phi / np.sqrt(np.sum(phi * phi))
    if phi[np.argmax(np.abs(phi))] < 0:
        phi = -phi
    return phi, float(np.sqrt(max(w[j], 0.0)))


@dataclasses.dataclass
class FdfdSpec:
    name: str
    n: int  # grid n x n (or n x ny when ny is set)
    npml: int
    eps_bg: float
    design: tuple  # (x0, y0, dx, dy) in cells
    eps_off: complex
    eps_on: complex
    slab: Optional[tuple] = None  # (y0, y1, eps) slab along x (interrupted by the design)
    source: str = "line"  # "line" (uniform Jz) or "mode"
    source_x: int = 13
    source_y: tuple = (10, 54)
    ports_x: tuple = (16, 50)
    port_kind: str = "line"  # "line" uniform average over source_y, or "mode" overlap
    norm: str = "incident"  # "incident" (empty-design fields) or "reference" (unbroken guide)
    obj_kind: int = OBJ_MAX_WEIGHTED_POWER
    obj_weights: tuple = (0.0, 1.0)
    ny: Optional[int] = None  # grid extent along y (default n)
    npml_y: Optional[int] = None  # PML along y (default npml; 0 = Dirichlet walls)
    lambda_cells: float = LAMBDA_CELLS  # free-space wavelength in cells (one frequency)


def _at_wavelength(spec: "FdfdSpec", lam: float) -> "FdfdSpec":
    return dataclasses.replace(spec, name=f"{spec.name}_l{lam:g}", lambda_cells=float(lam))


SPECS = {
    # 64^2, 10-cell PML, free space, line source, two monitor lines, 10x10 design in {1, 4}
    "fdfd64": FdfdSpec("fdfd64", 64, 10, 1.0, (27, 27, 10, 10), 1.0, 4.0,
                       source="line", source_x=13, source_y=(10, 54), ports_x=(16, 50),
                       port_kind="line", norm="incident"),
    # 128^2, 12-cell PML, eps=2.2 slab waveguide interrupted by a 32x32 design in {air, lossy metal}
    "fdfd128_metal": FdfdSpec("fdfd128_metal", 128, 12, 1.0, (48, 48, 32, 32), 1.0, 1.0 + 1e4j,
                              slab=(58, 70, 2.2), source="mode", source_x=16, ports_x=(20, 108),
                              port_kind="mode", norm="reference"),
    # 256^2, 16-cell PML, eps=2.2 slab interrupted by a 64x64 design in {1, 10}
    "fdfd256": FdfdSpec("fdfd256", 256, 16, 1.0, (96, 96, 64, 64), 1.0, 10.0,
                        slab=(120, 136, 2.2), source="mode", source_x=20, ports_x=(24, 232),
                        port_kind="mode", norm="reference"),
}
# the free-space device at two more frequencies (wavelengths of 19 and 21 cells):
# the systems of a multi-frequency design on one shared pixel layout
SPECS["fdfd64_l19"] = _at_wavelength(SPECS["fdfd64"], 19)
SPECS["fdfd64_l21"] = _at_wavelength(SPECS["fdfd64"], 21)
SPECS["fdfd128_metal_l19"] = _at_wavelength(SPECS["fdfd128_metal"], 19)
SPECS["fdfd128_metal_l21"] = _at_wavelength(SPECS["fdfd128_metal"], 21)


def _ny(spec: FdfdSpec) -> int:
    return spec.n if spec.ny is None else spec.ny


def _eps_grid(spec: FdfdSpec, with_slab_through_design: bool = False):
    eps = np.full((spec.n, _ny(spec)), spec.eps_bg, dtype=np.complex128)
    if spec.slab is not None:
        y0, y1, e = spec.slab
        eps[:, y0:y1] = e
    x0, y0, ddx, ddy = spec.design
    if not with_slab_through_design:
        eps[x0:x0 + ddx, y0:y0 + ddy] = spec.eps_off
    return eps


def _design_nodes(spec: FdfdSpec):
    x0, y0, ddx, ddy = spec.design
    ix, iy = np.meshgrid(np.arange(x0, x0 + ddx), np.arange(y0, y0 + ddy), indexing="ij")
    return (ix * _ny(spec) + iy).ravel()  # raster order: k = (ix-x0)*ddy + (iy-y0)


def _k(spec: FdfdSpec) -> float:
    return 2.0 * np.pi / spec.lambda_cells


def _source_and_ports(spec: FdfdSpec, eps: np.ndarray):
    n, ny = spec.n, _ny(spec)
    s = np.zeros((n, ny), dtype=np.complex128)
    ports = np.zeros((len(spec.ports_x), n, ny), dtype=np.complex128)
    if spec.source == "line":
        y0, y1 = spec.source_y
        s[spec.source_x, y0:y1] = 1.0
    else:
        phi, _ = slab_mode(eps[spec.source_x, :], _k(spec))
        s[spec.source_x, :] = phi
    for p, xp in enumerate(spec.ports_x):
        if spec.port_kind == "line":
            y0, y1 = spec.source_y
            ports[p, xp, y0:y1] = 1.0 / (y1 - y0)
        else:
            phi, _ = slab_mode(eps[xp, :], _k(spec))
            ports[p, xp, :] = phi
    return s.ravel(), ports.reshape(len(spec.ports_x), -1)


def solve_full(spec: FdfdSpec, eps: np.ndarray):
    """Direct sparse solve of the full structure: returns (E, port amplitudes)."""
    import scipy.sparse.linalg as spl

    A, sxy = helmholtz_operator(eps, spec.npml, _k(spec), npml_y=spec.npml_y)
    s, Pi = _source_and_ports(spec, _eps_grid(spec))
    E = spl.splu(A.tocsc()).solve(-(sxy * s))
    return E, Pi @ E


def make_fdfd_case(name, cache: bool = True) -> Case:
    """Build an FDFD workload by name (see ``SPECS``) or from an ``FdfdSpec``."""
    spec = SPECS[name] if isinstance(name, str) else name
    name = spec.name
    key = hashlib.sha1((json.dumps(dataclasses.asdict(spec), default=str) + RECIPE_VERSION).encode()).hexdigest()[:12]
    path = _cache_path(f"{name}_{key}.npz") if cache else None
    if path and os.path.exists(path):
        return _load_case(path)
    case = _build_fdfd(spec)
    if path:
        _save_case(path, case)
    return case


def _build_fdfd(spec: FdfdSpec) -> Case:
    import scipy.linalg as sla
    import scipy.sparse.linalg as spl

    n = spec.n * _ny(spec)
    k = _k(spec)
    eps = _eps_grid(spec)
    A, sxy = helmholtz_operator(eps, spec.npml, k, npml_y=spec.npml_y)
    dnodes = _design_nodes(spec)
    n_d = len(dnodes)
    mask = np.zeros(n, dtype=bool)
    mask[dnodes] = True
    rnodes = np.flatnonzero(~mask)
    A = A.tocsc()
    A_rr = A[rnodes][:, rnodes].tocsc()
    A_rd = A[rnodes][:, dnodes].tocsc()
    A_dd = A[dnodes][:, dnodes].toarray()
    # only design pixels on the region boundary couple to the rest
    bcols = np.flatnonzero(np.asarray(abs(A_rd).sum(axis=0)).ravel() > 0)
    lu_rr = spl.splu(A_rr)
    Z = lu_rr.solve(A_rd[:, bcols].toarray())  # (n_r, n_b)
    S = A_dd.copy()
    S[:, bcols] -= A_rd.T.tocsr() @ Z  # A_dr = A_rd^T
    # (A^-1)_dd = S^-1 and G = -(A^-1)_dd
    G = -sla.solve(S, np.eye(n_d, dtype=np.complex128), check_finite=False)
    G = 0.5 * (G + G.T)  # exact symmetry of a reciprocal medium (rounding only)
    # incident field and port functionals from the full background operator
    lu = spl.splu(A)
    s, Pi = _source_and_ports(spec, eps)
    E_inc = lu.solve(-(sxy * s))
    c_d = E_inc[dnodes].copy()
    c_o = Pi @ E_inc
    # G_od = -Pi^T A^-1 B = -(A^-1 Pi)^T B since A = A^T
    adj = lu.solve(np.ascontiguousarray(Pi.T))  # (n_nodes, n_o)
    G_od = -np.ascontiguousarray(adj[dnodes, :].T)
    dv = np.full(n_d, k * k * (spec.eps_on - spec.eps_off), dtype=np.complex128)
    if spec.norm == "incident":
        # the empty-design field at every port: the source-side port reports the
        # scattered part (S11 = (o_1 - c_o,1)/c_o,1), every other port the total
        # transmitted field (T_p1 = o_p/c_o,p)
        s_off = np.array([c_o[0]] + [0.0] * (len(c_o) - 1), dtype=np.complex128)
        s_scale = 1.0 / c_o
    else:
        # reference: the same source in the unbroken waveguide gives the incident mode amplitude
        eps_ref = _eps_grid(spec, with_slab_through_design=True)
        A_ref, _ = helmholtz_operator(eps_ref, spec.npml, k, npml_y=spec.npml_y)
        E_ref = spl.splu(A_ref.tocsc()).solve(-(sxy * s))
        a = Pi @ E_ref
        s_off = np.array([a[0]] + [0.0] * (len(a) - 1), dtype=np.complex128)
        s_scale = 1.0 / a
    meta = dict(kind="fdfd", spec=dataclasses.asdict(spec), k=k, n_boundary=len(bcols))
    return Case(spec.name, np.ascontiguousarray(G), G_od, c_d, c_o, dv, s_off, s_scale,
                spec.obj_kind, np.asarray(spec.obj_weights, dtype=np.float64), meta)


# ----------------------------------------------------------------------------
# Closed-form 2D Green function (homogeneous background)
# ----------------------------------------------------------------------------

def hankel_self_term(k: float = K_CELL) -> complex:
    """Cell-averaged self term: integral of (i/4) H0(k r) over an equal-area disk.

    With a = 1/sqrt(pi) (unit cell area), the integral is
    i*pi*a*H1(k a)/(2k) - 1/k^2.
    """
    from scipy.special import hankel1

    a = 1.0 / np.sqrt(np.pi)
    return complex(1j * np.pi * a * hankel1(1, k * a) / (2.0 * k) - 1.0 / (k * k))


def make_hankel_case(side: int = 128, n_ports: int = 4, ring_radius_lambda: float = 2.0,
                     eps_off: float = 1.0, eps_on: float = 4.0, name: Optional[str] = None,
                     cache: bool = True) -> Case:
    """Homogeneous 2D background, G_ij = (i/4) H0(k |r_i - r_j|) (cell area 1).

    Design: side x side pixels at integer coordinates; ports: points on a ring
    of the given radius centred on the design square, at 45 + 90 j degrees,
    snapped to cell corners; incident plane wave exp(i k x); objective:
    maximise |o_0|^2 normalised by the incident amplitude.
    """
    from scipy.special import hankel1

    name = name or f"hankel{side}"
    key = f"{name}_{side}_{n_ports}_{ring_radius_lambda}_{eps_off}_{eps_on}_{RECIPE_VERSION}"
    path = _cache_path(hashlib.sha1(key.encode()).hexdigest()[:12] + f"_{name}.npz") if cache else None
    if path and os.path.exists(path):
        return _load_case(path)
    k = K_CELL
    n_d = side * side
    # Toeplitz-block-Toeplitz: G depends only on (|dx|, |dy|)
    off = np.arange(side, dtype=np.float64)
    r = np.sqrt(off[:, None] ** 2 + off[None, :] ** 2)
    table = np.empty((side, side), dtype=np.complex128)
    nz = r > 0
    table[nz] = 0.25j * hankel1(0, k * r[nz])
    table[0, 0] = hankel_self_term(k)
    ix = np.repeat(np.arange(side), side)
    iy = np.tile(np.arange(side), side)
    G = np.empty((n_d, n_d), dtype=np.complex128)
    for i0 in range(0, n_d, 1024):
        i1 = min(n_d, i0 + 1024)
        G[i0:i1] = table[np.abs(ix[i0:i1, None] - ix[None, :]), np.abs(iy[i0:i1, None] - iy[None, :])]
    c = (side - 1) / 2.0
    rad = ring_radius_lambda * LAMBDA_CELLS
    ang = np.deg2rad(45.0 + 90.0 * np.arange(n_ports))
    px = np.floor(c + rad * np.cos(ang)) + 0.5
    py = np.floor(c + rad * np.sin(ang)) + 0.5
    rp = np.sqrt((px[:, None] - ix[None, :]) ** 2 + (py[:, None] - iy[None, :]) ** 2)
    G_od = 0.25j * hankel1(0, k * rp)
    c_d = np.exp(1j * k * ix).astype(np.complex128)
    c_o = np.exp(1j * k * px).astype(np.complex128)
    dv = np.full(n_d, k * k * (eps_on - eps_off), dtype=np.complex128)
    w = np.zeros(n_ports); w[0] = 1.0
    meta = dict(kind="hankel", side=side, ports=np.stack([px, py], 1).tolist(), k=k)
    case = Case(name, G, np.ascontiguousarray(G_od), c_d, c_o, dv, np.zeros(n_ports, np.complex128),
                1.0 / c_o, OBJ_MAX_WEIGHTED_POWER, w, meta)
    if path:
        _save_case(path, case)
    return case


# ----------------------------------------------------------------------------
# Seeded designs and visiting orders
# ----------------------------------------------------------------------------

def random_design(n_d: int, seed: int, p: float = 0.5) -> np.ndarray:
    """b_0 ~ Bernoulli(p) per pixel, numpy PCG64(seed); uint8."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return (rng.random(n_d) < p).astype(np.uint8)


def square_tiles(side_x: int, side_y: int, t: int) -> np.ndarray:
    """Tiles of t x t pixels over a side_x x side_y region in raster order
    (pixel k = x * side_y + y); (side_x/t * side_y/t, t*t) int32."""
    assert side_x % t == 0 and side_y % t == 0
    out = []
    for tx in range(side_x // t):
        for ty in range(side_y // t):
            out.append([(tx * t + i) * side_y + ty * t + j for i in range(t) for j in range(t)])
    return np.asarray(out, dtype=np.int32)


def mirror_tied_tiles(side_x: int, side_y: int, t: int) -> np.ndarray:
    """t x t tiles tied to their mirror image about the region's centre line
    y -> side_y - 1 - y (a design kept symmetric, as the paper's designs flip 2
    or 4 symmetry-tied tiles at once); a tile on the centre line is its own
    image and is padded with -1.  Shape (n_tied, 2*t*t) int32."""
    sq = square_tiles(side_x, side_y, t)
    nty = side_y // t
    out = []
    for tx in range(side_x // t):
        for ty in range((nty + 1) // 2):
            a = sq[tx * nty + ty]
            m = nty - 1 - ty
            if m == ty:
                out.append(np.concatenate([a, -np.ones_like(a)]))
            else:
                out.append(np.concatenate([a, sq[tx * nty + m]]))
    return np.asarray(out, dtype=np.int32)


def raster_order(n_d: int, n_sweeps: int) -> np.ndarray:
    return np.tile(np.arange(n_d, dtype=np.int32), (n_sweeps, 1))


def shuffled_order(n_d: int, n_sweeps: int, seed: int) -> np.ndarray:
    """One seeded permutation per sweep (PCG64 seeded with (seed, sweep))."""
    out = np.empty((n_sweeps, n_d), dtype=np.int32)
    for s in range(n_sweeps):
        rng = np.random.Generator(np.random.PCG64([seed, s]))
        out[s] = rng.permutation(n_d).astype(np.int32)
    return out


# ----------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------

WORKLOADS = {
    "fdfd64_nd100": dict(case="fdfd64", n_sweeps=3, seed=0),
    "fdfd128_metal_nd1024": dict(case="fdfd128_metal", n_sweeps=10, seed=0),
    "fdfd256_nd4096": dict(case="fdfd256", n_sweeps=3, seed=0),
}


def get_case(name: str) -> Case:
    if name.startswith("hankel"):
        side = int(name[len("hankel"):] or 128)
        # a large closed-form G is faster to rebuild (~15 s at 128 x 128) than to cache (4.3 GB)
        return make_hankel_case(side, cache=side <= 64)
    return make_fdfd_case(name)


def _cache_path(fname: str) -> Optional[str]:
    """Cache file for generated inputs: $PNGF_CACHE_DIR, else pngf_cache in the
    system's temporary directory; PNGF_CACHE_DIR=off disables the cache."""
    d = os.environ.get("PNGF_CACHE_DIR") or os.path.join(tempfile.gettempdir(), "pngf_cache")
    if d in ("", "0", "off"):
        return None
    os.makedirs(d, exist_ok=True)
    return os.path.join(d, fname)


def _save_case(path: str, case: Case) -> None:
    tmp = path + f".tmp{os.getpid()}.npz"
    np.savez(tmp, G_dd=case.G_dd, G_od=case.G_od, c_d=case.c_d, c_o=case.c_o, dv=case.dv,
             s_off=case.s_off, s_scale=case.s_scale, obj_weights=case.obj_weights,
             obj_kind=np.int64(case.obj_kind), name=np.str_(case.name),
             meta=np.str_(json.dumps(case.meta, default=str)))
    os.replace(tmp, path)


def _load_case(path: str) -> Case:
    z = np.load(path)
    return Case(str(z["name"]), z["G_dd"], z["G_od"], z["c_d"], z["c_o"], z["dv"], z["s_off"],
                z["s_scale"], int(z["obj_kind"]), z["obj_weights"], json.loads(str(z["meta"])))
