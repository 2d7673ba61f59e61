"""Thin ctypes binding of the C ABI in include/pngf.h (argument marshalling only).

Every function below has the name of the C entry point it calls and forwards
plain integers / device pointers; all arithmetic of the hot path runs in the
CUDA kernels of ``libpngf.so``.  ``DbsContext`` is a convenience wrapper that
keeps the torch tensors (device memory) alive for one context.

The library is loaded from this package directory; if it is missing the import
of the binding functions fails loudly (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpngf.so")

PNGF_OK, PNGF_EINVAL, PNGF_ENOMEM, PNGF_ECUDA, PNGF_ESINGULAR = 0, 1, 2, 3, 4
PNGF_ENOTFACTORED, PNGF_ETIMEOUT, PNGF_ENUMERIC, PNGF_ECAPACITY, PNGF_EACCURACY = 5, 6, 7, 8, 9
PNGF_FP64, PNGF_MIXED, PNGF_PEC = 0, 1, 2
PNGF_FIRST_IMPROVEMENT, PNGF_BEST_IMPROVEMENT = 0, 1
PNGF_OBJ_MAX_WEIGHTED_POWER, PNGF_OBJ_MIN_INSERTION_LOSS = 0, 1
PNGF_MAX_PORTS = 8
PNGF_NOALLOC_MAX_ND = 8192
PNGF_BATCH_MAX_RUNS = 65536
PNGF_BATCH_MAX_ND = 4096
PNGF_TILES_MAX_SYSTEMS, PNGF_TILE_MAX = 4, 16
PNGF_COMBINE_MEAN, PNGF_COMBINE_WORST = 0, 1


class pngf_config(ctypes.Structure):
    _fields_ = [
        ("n_d", ctypes.c_int32),
        ("n_o", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("mode", ctypes.c_int32),
        ("objective", ctypes.c_int32),
        ("refresh_k", ctypes.c_int32),
        ("delay_r", ctypes.c_int32),
        ("n_ctas", ctypes.c_int32),
        ("tau", ctypes.c_double),
        ("obj_weights", ctypes.c_double * PNGF_MAX_PORTS),
        ("s_off", ctypes.c_double * (2 * PNGF_MAX_PORTS)),
        ("s_scale", ctypes.c_double * (2 * PNGF_MAX_PORTS)),
        ("tensor_fold", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class PngfError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {pngf_status_string(status)} (status {status})")
        self.status = status


_lib = None
_P = ctypes.c_void_p


def lib() -> ctypes.CDLL:
    """Load libpngf.so (built by ``paper_2501_18054_gb300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                               "(python -m paper_2501_18054_gb300.build)")
        L = ctypes.CDLL(LIB_PATH)
        st = ctypes.c_int
        sig = {
            "pngf_workspace_size": (st, [ctypes.POINTER(pngf_config), ctypes.POINTER(ctypes.c_size_t)]),
            "pngf_create": (st, [ctypes.POINTER(pngf_config), _P, _P, _P, _P, _P, _P, ctypes.c_size_t, _P,
                                 ctypes.POINTER(_P)]),
            "pngf_factor": (st, [_P, _P]),
            "pngf_score_flips": (st, [_P, _P, ctypes.c_int32, _P, _P]),
            "pngf_accept_flip": (st, [_P, ctypes.c_int32]),
            "pngf_accept_flip_noalloc": (st, [_P, ctypes.c_int32]),
            "pngf_dbs_sweep": (st, [_P, ctypes.c_int32, _P, _P, _P, ctypes.c_int32, _P]),
            "pngf_batch_workspace_size": (st, [ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]),
            "pngf_dbs_sweep_batch": (st, [_P, ctypes.c_int32, ctypes.c_int32, _P, _P, _P, ctypes.c_int32, _P, _P,
                                          ctypes.c_size_t]),
            "pngf_eval_ports": (st, [_P, _P, _P]),
            "pngf_get_design": (st, [_P, _P]),
            "pngf_get_state": (st, [_P, _P, _P, _P, _P, _P]),
            "pngf_gradient": (st, [_P, _P, _P]),
            "pngf_set_launch": (st, [_P, ctypes.c_int32, ctypes.c_int32]),
            "pngf_tiles_workspace_size": (st, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                               ctypes.POINTER(ctypes.c_size_t)]),
            "pngf_dbs_sweep_tiles": (st, [_P, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_int32, _P, _P, _P, ctypes.c_int32, _P, _P, ctypes.c_size_t]),
            "pngf_score_tiles": (st, [_P, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int32, ctypes.c_int32, _P,
                                      ctypes.c_int32, _P, _P, _P, ctypes.c_size_t]),
            "pngf_accept_tile": (st, [_P, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_int32, _P, ctypes.c_size_t]),
            "pngf_get_since_refresh": (st, [_P, _P]),
            "pngf_set_state": (st, [_P, _P, _P, _P, _P, _P, _P, ctypes.c_int32]),
            "pngf_set_wait_limit": (st, [_P, ctypes.c_int32, ctypes.c_int32]),
            "pngf_snapshot": (st, [_P]),
            "pngf_restore": (st, [_P]),
            "pngf_sync": (st, [_P]),
            "pngf_get_phase_cycles": (st, [_P, _P]),
            "pngf_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "pngf_destroy": (None, [_P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols() -> list:
    """Names of the pngf_* entry points the loaded library resolves."""
    L = lib()
    names = []
    for n in ("pngf_workspace_size", "pngf_create", "pngf_factor", "pngf_score_flips", "pngf_accept_flip",
              "pngf_accept_flip_noalloc", "pngf_batch_workspace_size", "pngf_dbs_sweep_batch",
              "pngf_dbs_sweep", "pngf_eval_ports", "pngf_get_design", "pngf_get_state",
              "pngf_gradient", "pngf_set_launch", "pngf_tiles_workspace_size", "pngf_dbs_sweep_tiles", "pngf_score_tiles",
              "pngf_accept_tile", "pngf_get_since_refresh", "pngf_set_state", "pngf_set_wait_limit", "pngf_snapshot",
              "pngf_restore", "pngf_sync", "pngf_get_phase_cycles", "pngf_status_string", "pngf_destroy"):
        if hasattr(L, n):
            names.append(n)
    return names


def _check(status: int, where: str) -> None:
    if status != PNGF_OK:
        raise PngfError(status, where)


# ---------------------------------------------------------------- 1:1 entry points
def pngf_status_string(status: int) -> str:
    return lib().pngf_status_string(int(status)).decode()


def pngf_workspace_size(cfg: pngf_config) -> int:
    out = ctypes.c_size_t(0)
    _check(lib().pngf_workspace_size(ctypes.byref(cfg), ctypes.byref(out)), "pngf_workspace_size")
    return int(out.value)


def pngf_create(cfg: pngf_config, G_dd: int, G_od: int, c_d: int, c_o: int, dv: int, workspace: int,
                workspace_bytes: int, stream: int) -> int:
    h = _P()
    _check(lib().pngf_create(ctypes.byref(cfg), G_dd, G_od, c_d, c_o, dv, workspace, workspace_bytes,
                             stream, ctypes.byref(h)), "pngf_create")
    return h.value


def pngf_factor(ctx: int, b: int) -> None:
    _check(lib().pngf_factor(ctx, b), "pngf_factor")


def pngf_score_flips(ctx: int, pixels: int, n: int, f_new: int, o_new: Optional[int]) -> None:
    _check(lib().pngf_score_flips(ctx, pixels, n, f_new, o_new), "pngf_score_flips")


def pngf_accept_flip(ctx: int, pixel: int) -> None:
    _check(lib().pngf_accept_flip(ctx, int(pixel)), "pngf_accept_flip")


def pngf_accept_flip_noalloc(ctx: int, pixel: int) -> None:
    _check(lib().pngf_accept_flip_noalloc(ctx, int(pixel)), "pngf_accept_flip_noalloc")


def pngf_dbs_sweep(ctx: int, n_sweeps: int, order: Optional[int], trace: Optional[int],
                   trace_f: Optional[int], trace_cap: int, counters: Optional[int]) -> None:
    _check(lib().pngf_dbs_sweep(ctx, n_sweeps, order, trace, trace_f, trace_cap, counters), "pngf_dbs_sweep")


def pngf_batch_workspace_size(n_ctx: int) -> int:
    out = ctypes.c_size_t(0)
    _check(lib().pngf_batch_workspace_size(int(n_ctx), ctypes.byref(out)), "pngf_batch_workspace_size")
    return int(out.value)


def _ptr_array(ptrs):
    if ptrs is None:
        return None
    arr = (ctypes.c_void_p * len(ptrs))(*[p if p else None for p in ptrs])
    return arr


def pngf_dbs_sweep_batch(ctxs, n_sweeps: int, orders, traces, trace_f, trace_cap: int, counters: Optional[int],
                         batch_ws: int, batch_ws_bytes: int) -> None:
    h = (ctypes.c_void_p * len(ctxs))(*ctxs)
    o, t, tf = _ptr_array(orders), _ptr_array(traces), _ptr_array(trace_f)
    _check(lib().pngf_dbs_sweep_batch(ctypes.cast(h, _P), len(ctxs), int(n_sweeps),
                                      ctypes.cast(o, _P) if o is not None else None,
                                      ctypes.cast(t, _P) if t is not None else None,
                                      ctypes.cast(tf, _P) if tf is not None else None,
                                      int(trace_cap), counters, batch_ws, int(batch_ws_bytes)),
           "pngf_dbs_sweep_batch")


def pngf_eval_ports(ctx: int, n_o: int):
    o = (ctypes.c_double * (2 * n_o))()
    f = ctypes.c_double(0.0)
    _check(lib().pngf_eval_ports(ctx, ctypes.cast(o, _P), ctypes.cast(ctypes.byref(f), _P)), "pngf_eval_ports")
    arr = np.frombuffer(o, dtype=np.float64).copy()
    return arr[0::2] + 1j * arr[1::2], float(f.value)


def pngf_get_design(ctx: int, b: int) -> None:
    _check(lib().pngf_get_design(ctx, b), "pngf_get_design")


def pngf_get_state(ctx: int, W: Optional[int], diag_W: Optional[int], e: Optional[int], T: Optional[int],
                   o: Optional[int]) -> None:
    _check(lib().pngf_get_state(ctx, W, diag_W, e, T, o), "pngf_get_state")


def pngf_gradient(ctx: int, grad: int, dodrho: Optional[int]) -> None:
    _check(lib().pngf_gradient(ctx, grad, dodrho), "pngf_gradient")


def pngf_tiles_workspace_size(n_sys: int, n_d: int, n_tiles: int, tile_m: int) -> int:
    out = ctypes.c_size_t(0)
    _check(lib().pngf_tiles_workspace_size(int(n_sys), int(n_d), int(n_tiles), int(tile_m), ctypes.byref(out)),
           "pngf_tiles_workspace_size")
    return int(out.value)


def _ctx_array(ctxs):
    h = (ctypes.c_void_p * len(ctxs))(*ctxs)
    return h, ctypes.cast(h, _P)


def pngf_dbs_sweep_tiles(ctxs, combine: int, tiles: int, n_tiles: int, tile_m: int, n_sweeps: int,
                         order: Optional[int], trace: Optional[int], trace_f: Optional[int], trace_cap: int,
                         counters: Optional[int], ws: int, ws_bytes: int) -> None:
    h, hp = _ctx_array(ctxs)
    _check(lib().pngf_dbs_sweep_tiles(hp, len(ctxs), int(combine), tiles, int(n_tiles), int(tile_m), int(n_sweeps),
                                      order, trace, trace_f, int(trace_cap), counters, ws, int(ws_bytes)),
           "pngf_dbs_sweep_tiles")


def pngf_score_tiles(ctxs, combine: int, tiles: int, n_tiles: int, tile_m: int, lst: int, count: int, F: int,
                     f_sys: Optional[int], ws: int, ws_bytes: int) -> None:
    h, hp = _ctx_array(ctxs)
    _check(lib().pngf_score_tiles(hp, len(ctxs), int(combine), tiles, int(n_tiles), int(tile_m), lst, int(count), F,
                                  f_sys, ws, int(ws_bytes)), "pngf_score_tiles")


def pngf_accept_tile(ctxs, combine: int, tiles: int, n_tiles: int, tile_m: int, tile: int, ws: int,
                     ws_bytes: int) -> None:
    h, hp = _ctx_array(ctxs)
    _check(lib().pngf_accept_tile(hp, len(ctxs), int(combine), tiles, int(n_tiles), int(tile_m), int(tile), ws,
                                  int(ws_bytes)), "pngf_accept_tile")


def pngf_set_launch(ctx: int, n_ctas: int, tensor_fold: int) -> None:
    _check(lib().pngf_set_launch(ctx, int(n_ctas), int(tensor_fold)), "pngf_set_launch")


def pngf_get_since_refresh(ctx: int) -> int:
    out = ctypes.c_int32(0)
    _check(lib().pngf_get_since_refresh(ctx, ctypes.cast(ctypes.byref(out), _P)), "pngf_get_since_refresh")
    return int(out.value)


def pngf_set_state(ctx: int, b: Optional[int], W: Optional[int], diag_W: int, e: int, T: int, o: int,
                   since_refresh: int) -> None:
    _check(lib().pngf_set_state(ctx, b, W, diag_W, e, T, o, int(since_refresh)), "pngf_set_state")


def pngf_set_wait_limit(ctx: int, wait_log2: int, hold_cta: int) -> None:
    _check(lib().pngf_set_wait_limit(ctx, int(wait_log2), int(hold_cta)), "pngf_set_wait_limit")


def pngf_snapshot(ctx: int) -> None:
    _check(lib().pngf_snapshot(ctx), "pngf_snapshot")


def pngf_restore(ctx: int) -> None:
    _check(lib().pngf_restore(ctx), "pngf_restore")


def pngf_get_phase_cycles(ctx: int) -> np.ndarray:
    out = (ctypes.c_int64 * 16)()
    _check(lib().pngf_get_phase_cycles(ctx, ctypes.cast(out, _P)), "pngf_get_phase_cycles")
    return np.frombuffer(out, dtype=np.int64).copy()


def pngf_sync(ctx: int) -> int:
    return int(lib().pngf_sync(ctx))


def pngf_destroy(ctx: int) -> None:
    lib().pngf_destroy(ctx)


# ---------------------------------------------------------------- convenience wrapper
def make_config(n_d: int, n_o: int, *, precision: int = PNGF_FP64, mode: int = PNGF_FIRST_IMPROVEMENT,
                objective: int = PNGF_OBJ_MAX_WEIGHTED_POWER, refresh_k: int = 64, delay_r: int = 64,
                n_ctas: int = 0, tau: float = 1e-9, obj_weights=None, s_off=None, s_scale=None,
                tensor_fold: int = 0) -> pngf_config:
    cfg = pngf_config()
    cfg.n_d, cfg.n_o = int(n_d), int(n_o)
    cfg.precision, cfg.mode, cfg.objective = int(precision), int(mode), int(objective)
    cfg.refresh_k, cfg.delay_r, cfg.n_ctas, cfg.tau = int(refresh_k), int(delay_r), int(n_ctas), float(tau)
    cfg.tensor_fold = int(tensor_fold)
    w = np.zeros(PNGF_MAX_PORTS)
    if obj_weights is not None:
        w[:n_o] = np.asarray(obj_weights, dtype=np.float64)[:n_o]
    off = np.zeros(PNGF_MAX_PORTS, dtype=np.complex128)
    sc = np.ones(PNGF_MAX_PORTS, dtype=np.complex128)
    if s_off is not None:
        off[:n_o] = np.asarray(s_off, dtype=np.complex128)[:n_o]
    if s_scale is not None:
        sc[:n_o] = np.asarray(s_scale, dtype=np.complex128)[:n_o]
    for p in range(PNGF_MAX_PORTS):
        cfg.obj_weights[p] = w[p]
        cfg.s_off[2 * p], cfg.s_off[2 * p + 1] = off[p].real, off[p].imag
        cfg.s_scale[2 * p], cfg.s_scale[2 * p + 1] = sc[p].real, sc[p].imag
    return cfg


class DbsContext:
    """One design region on one GPU: owns the torch tensors behind the C context."""

    def __init__(self, case, *, precision: int = PNGF_FP64, mode: int = PNGF_FIRST_IMPROVEMENT,
                 tau: float = 1e-9, refresh_k: int = 64, delay_r: int = 64, n_ctas: int = 0,
                 device: str = "cuda", stream=None, inputs_on_device=None, tensor_fold: int = 0):
        import torch

        self.torch = torch
        self.n_d, self.n_o = case.n_d, case.n_o
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)

        def dev(x):
            t = x if isinstance(x, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(x))
            return t.to(self.device, dtype=torch.complex128).contiguous()

        if inputs_on_device is not None:
            self.G, self.God, self.cd, self.co, self.dv = inputs_on_device
        else:
            self.G, self.God, self.cd, self.co, self.dv = (dev(case.G_dd), dev(case.G_od), dev(case.c_d),
                                                           dev(case.c_o), dev(case.dv))
        self.cfg = make_config(case.n_d, case.n_o, precision=precision, mode=mode, objective=case.obj_kind,
                               refresh_k=refresh_k, delay_r=delay_r, n_ctas=n_ctas, tau=tau,
                               obj_weights=case.obj_weights, s_off=case.s_off, s_scale=case.s_scale,
                               tensor_fold=tensor_fold)
        self.ws_bytes = pngf_workspace_size(self.cfg)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        self.ctx = pngf_create(self.cfg, self.G.data_ptr(), self.God.data_ptr(), self.cd.data_ptr(),
                               self.co.data_ptr(), self.dv.data_ptr(), self.ws.data_ptr(), self.ws_bytes,
                               self.stream.cuda_stream)
        self.counters = torch.zeros(8, dtype=torch.int64, device=self.device)

    # -- calls
    def factor(self, b) -> None:
        bt = self.torch.as_tensor(np.asarray(b, dtype=np.uint8)).to(self.device) if not isinstance(
            b, self.torch.Tensor) else b.to(self.device, self.torch.uint8)
        self._b_keep = bt
        pngf_factor(self.ctx, bt.data_ptr())

    def score_flips(self, pixels, want_ports: bool = False):
        torch = self.torch
        px = torch.as_tensor(np.asarray(pixels, dtype=np.int32)).to(self.device)
        f = torch.empty(len(px), dtype=torch.float64, device=self.device)
        o = torch.empty((len(px), self.n_o), dtype=torch.complex128, device=self.device) if want_ports else None
        pngf_score_flips(self.ctx, px.data_ptr(), len(px), f.data_ptr(), o.data_ptr() if o is not None else None)
        self.stream.synchronize()
        return (f.cpu().numpy(), o.cpu().numpy()) if want_ports else f.cpu().numpy()

    def accept_flip(self, pixel: int) -> None:
        pngf_accept_flip(self.ctx, pixel)

    def dbs_sweep(self, n_sweeps: int, order=None, trace_cap: Optional[int] = None, sync: bool = True):
        torch = self.torch
        if trace_cap is None:
            trace_cap = max(1, n_sweeps * self.n_d)
        od = None
        if order is not None:
            od = order if isinstance(order, torch.Tensor) else torch.as_tensor(
                np.ascontiguousarray(order, dtype=np.int32))
            od = od.to(self.device, torch.int32).contiguous()
        self._order_keep = od
        self.trace = torch.zeros((trace_cap, 4), dtype=torch.int32, device=self.device)
        self.trace_f = torch.zeros(trace_cap, dtype=torch.float64, device=self.device)
        pngf_dbs_sweep(self.ctx, n_sweeps, od.data_ptr() if od is not None else None, self.trace.data_ptr(),
                       self.trace_f.data_ptr(), trace_cap, self.counters.data_ptr())
        if not sync:
            return None
        st = pngf_sync(self.ctx)
        if st not in (PNGF_OK,):
            raise PngfError(st, "pngf_dbs_sweep")
        c = self.counters.cpu().numpy()
        n_acc = int(min(c[0], trace_cap))
        return dict(trace=self.trace[:n_acc].cpu().numpy(), trace_f=self.trace_f[:n_acc].cpu().numpy(),
                    counters=c)

    def eval_ports(self):
        return pngf_eval_ports(self.ctx, self.n_o)

    def design(self) -> np.ndarray:
        b = self.torch.empty(self.n_d, dtype=self.torch.uint8, device=self.device)
        pngf_get_design(self.ctx, b.data_ptr())
        self.stream.synchronize()
        return b.cpu().numpy()

    def state(self, with_W: bool = False) -> dict:
        torch = self.torch
        n, n_o = self.n_d, self.n_o
        W = torch.empty((n, n), dtype=torch.complex128, device=self.device) if with_W else None
        d = torch.empty(n, dtype=torch.complex128, device=self.device)
        e = torch.empty(n, dtype=torch.complex128, device=self.device)
        T = torch.empty((n_o, n), dtype=torch.complex128, device=self.device)
        o = torch.empty(n_o, dtype=torch.complex128, device=self.device)
        pngf_get_state(self.ctx, W.data_ptr() if W is not None else None, d.data_ptr(), e.data_ptr(),
                       T.data_ptr(), o.data_ptr())
        self.stream.synchronize()
        out = dict(diag=d.cpu().numpy(), e=e.cpu().numpy(), T=T.cpu().numpy(), o=o.cpu().numpy())
        if W is not None:
            out["W"] = W.cpu().numpy()
        return out

    def gradient(self, want_dodrho: bool = False):
        """df/drho at the current design (pngf_gradient), as host arrays."""
        torch = self.torch
        g = torch.empty(self.n_d, dtype=torch.float64, device=self.device)
        d = torch.empty((self.n_o, self.n_d), dtype=torch.complex128, device=self.device) if want_dodrho else None
        pngf_gradient(self.ctx, g.data_ptr(), d.data_ptr() if d is not None else None)
        self.stream.synchronize()
        return (g.cpu().numpy(), d.cpu().numpy()) if want_dodrho else g.cpu().numpy()

    def checkpoint(self) -> dict:
        """The maintained state as host arrays (pngf_get_state / _design / _since_refresh)."""
        st = self.state(with_W=self.cfg.precision == PNGF_FP64)
        st["b"] = self.design()
        st["since_refresh"] = pngf_get_since_refresh(self.ctx)
        return st

    def set_state(self, ck: dict) -> None:
        """Import a checkpoint() (pngf_set_state); FP64 contexts take b and W too."""
        torch = self.torch
        fp64 = self.cfg.precision == PNGF_FP64

        def dev(x, dt):
            return torch.as_tensor(np.ascontiguousarray(x)).to(self.device, dt)

        keep = dict(d=dev(ck["diag"], torch.complex128), e=dev(ck["e"], torch.complex128),
                    T=dev(ck["T"], torch.complex128), o=dev(ck["o"], torch.complex128))
        if fp64:
            keep["W"] = dev(ck["W"], torch.complex128)
            keep["b"] = dev(ck["b"], torch.uint8)
        pngf_set_state(self.ctx, keep["b"].data_ptr() if fp64 else None, keep["W"].data_ptr() if fp64 else None,
                       keep["d"].data_ptr(), keep["e"].data_ptr(), keep["T"].data_ptr(), keep["o"].data_ptr(),
                       int(ck["since_refresh"]))
        self.stream.synchronize()

    def set_launch(self, n_ctas: int, tensor_fold: int) -> None:
        pngf_set_launch(self.ctx, n_ctas, tensor_fold)
        self.cfg.n_ctas, self.cfg.tensor_fold = int(n_ctas), int(tensor_fold)

    def set_wait_limit(self, wait_log2: int, hold_cta: int = -1) -> None:
        pngf_set_wait_limit(self.ctx, wait_log2, hold_cta)

    def phase_cycles(self) -> np.ndarray:
        return pngf_get_phase_cycles(self.ctx)

    def snapshot(self) -> None:
        pngf_snapshot(self.ctx)

    def restore(self) -> None:
        pngf_restore(self.ctx)

    def sync(self) -> int:
        return pngf_sync(self.ctx)

    def close(self) -> None:
        if getattr(self, "ctx", None):
            pngf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DbsBatch:
    """Many independent runs (one DbsContext each) advanced by one launch."""

    def __init__(self, contexts):
        import torch

        self.torch = torch
        self.ctxs = list(contexts)
        c0 = self.ctxs[0]
        self.device = c0.device
        self.stream = c0.stream
        self.ws_bytes = pngf_batch_workspace_size(len(self.ctxs))
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        self.counters = torch.zeros((len(self.ctxs), 8), dtype=torch.int64, device=self.device)

    def dbs_sweep(self, n_sweeps: int, orders=None, trace_cap: Optional[int] = None, sync: bool = True):
        torch = self.torch
        if trace_cap is None:
            trace_cap = max(1, n_sweeps * max(c.n_d for c in self.ctxs))
        self.traces = [torch.zeros((trace_cap, 4), dtype=torch.int32, device=self.device) for _ in self.ctxs]
        self.trace_fs = [torch.zeros(trace_cap, dtype=torch.float64, device=self.device) for _ in self.ctxs]
        od = None
        if orders is not None:
            self._orders_keep = [None if o is None else torch.as_tensor(np.ascontiguousarray(o, dtype=np.int32)).to(
                self.device) for o in orders]
            od = [0 if o is None else o.data_ptr() for o in self._orders_keep]
        pngf_dbs_sweep_batch([c.ctx for c in self.ctxs], n_sweeps, od, [t.data_ptr() for t in self.traces],
                             [t.data_ptr() for t in self.trace_fs], trace_cap, self.counters.data_ptr(),
                             self.ws.data_ptr(), self.ws_bytes)
        if not sync:
            return None
        for c in self.ctxs:
            st = c.sync()
            if st != PNGF_OK:
                raise PngfError(st, "pngf_dbs_sweep_batch")
        cnt = self.counters.cpu().numpy()
        out = []
        for i, c in enumerate(self.ctxs):
            n_acc = int(min(cnt[i, 0], trace_cap))
            out.append(dict(trace=self.traces[i][:n_acc].cpu().numpy(), trace_f=self.trace_fs[i][:n_acc].cpu().numpy(),
                            counters=cnt[i]))
        return out


class TileSearch:
    """DBS over tile flips on one or several systems (one DbsContext each, FP64,
    factored at the same design) that share the design: pngf_dbs_sweep_tiles."""

    def __init__(self, contexts, tiles, combine: int = PNGF_COMBINE_MEAN):
        import torch

        self.torch = torch
        self.ctxs = list(contexts)
        c0 = self.ctxs[0]
        self.device, self.stream = c0.device, c0.stream
        t = np.ascontiguousarray(np.asarray(tiles, dtype=np.int32))
        if t.ndim == 1:
            t = t[:, None]
        self.n_tiles, self.tile_m = t.shape
        self.tiles = torch.as_tensor(t).to(self.device)
        self.combine = int(combine)
        self.ws_bytes = pngf_tiles_workspace_size(len(self.ctxs), c0.n_d, self.n_tiles, self.tile_m)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        self.counters = torch.zeros(8, dtype=torch.int64, device=self.device)

    def _h(self):
        return [c.ctx for c in self.ctxs]

    def dbs_sweep(self, n_sweeps: int, order=None, trace_cap: Optional[int] = None, sync: bool = True):
        torch = self.torch
        if trace_cap is None:
            trace_cap = max(1, n_sweeps * self.n_tiles)
        od = None
        if order is not None:
            od = torch.as_tensor(np.ascontiguousarray(order, dtype=np.int32)).to(self.device)
        self._order_keep = od
        self.trace = torch.zeros((trace_cap, 4), dtype=torch.int32, device=self.device)
        self.trace_f = torch.zeros(trace_cap, dtype=torch.float64, device=self.device)
        pngf_dbs_sweep_tiles(self._h(), self.combine, self.tiles.data_ptr(), self.n_tiles, self.tile_m, n_sweeps,
                             od.data_ptr() if od is not None else None, self.trace.data_ptr(),
                             self.trace_f.data_ptr(), trace_cap, self.counters.data_ptr(), self.ws.data_ptr(),
                             self.ws_bytes)
        if not sync:
            return None
        st = self.ctxs[0].sync()
        if st != PNGF_OK:
            raise PngfError(st, "pngf_dbs_sweep_tiles")
        c = self.counters.cpu().numpy()
        n_acc = int(min(c[0], trace_cap))
        return dict(trace=self.trace[:n_acc].cpu().numpy(), trace_f=self.trace_f[:n_acc].cpu().numpy(), counters=c)

    def score(self, tiles_idx=None, per_system: bool = False):
        torch = self.torch
        idx = np.arange(self.n_tiles, dtype=np.int32) if tiles_idx is None else np.asarray(tiles_idx, np.int32)
        lst = torch.as_tensor(idx).to(self.device)
        F = torch.empty(len(idx), dtype=torch.float64, device=self.device)
        fs = torch.empty((len(idx), len(self.ctxs)), dtype=torch.float64, device=self.device) if per_system else None
        pngf_score_tiles(self._h(), self.combine, self.tiles.data_ptr(), self.n_tiles, self.tile_m, lst.data_ptr(),
                         len(idx), F.data_ptr(), fs.data_ptr() if fs is not None else None, self.ws.data_ptr(),
                         self.ws_bytes)
        self.stream.synchronize()
        return (F.cpu().numpy(), fs.cpu().numpy()) if per_system else F.cpu().numpy()

    def accept(self, tile: int) -> None:
        pngf_accept_tile(self._h(), self.combine, self.tiles.data_ptr(), self.n_tiles, self.tile_m, int(tile),
                         self.ws.data_ptr(), self.ws_bytes)
        st = self.ctxs[0].sync()
        if st != PNGF_OK:
            raise PngfError(st, "pngf_accept_tile")
