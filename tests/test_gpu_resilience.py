"""Failure detection, checkpoint / resume and graph capture through the C ABI.

* A bounded device wait that runs out: one CTA of a persistent sweep is held
  on a flag that nothing sets (pngf_set_wait_limit), the others' grid-barrier
  or word waits give up after a short limit and the call ends with
  PNGF_ETIMEOUT latched -- no fault, no hang -- and the same context then runs
  the search correctly again.
* A checkpoint exported from one context (pngf_get_state, pngf_get_design,
  pngf_get_since_refresh) and imported into a fresh context of the same inputs
  (pngf_set_state) resumes the search: on the FP64 path the resumed trajectory
  is bit for bit the uninterrupted one.
* One batched call (restore + pngf_dbs_sweep_batch) captured in a CUDA graph
  and replayed gives bit for bit the eager call's results.
"""
import json
import os

import numpy as np
import pytest

from paper_2501_18054_gb300 import workloads as W

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


def _golden(name):
    with open(os.path.join(HERE, "golden", name + ".json")) as fh:
        return json.load(fh)


def _seq(trace):
    return [tuple(int(x) for x in r[:3]) for r in trace]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_held_cta_times_out_then_context_recovers(P, fdfd64, precision):
    g = _golden("fdfd64_first_raster")
    kw = dict(tau=g["tau"], refresh_k=16)
    if precision == "mixed":
        kw.update(precision=P.PNGF_MIXED, delay_r=8, tensor_fold=1)
    ctx = P.DbsContext(fdfd64, **kw)
    ctx.factor(W.random_design(fdfd64.n_d, g["spec"]["seed"]))
    ctx.snapshot()
    ctx.set_wait_limit(14, hold_cta=1)  # 2^14 polls: milliseconds
    ctx.dbs_sweep(g["spec"]["n_sweeps"], sync=False)
    assert ctx.sync() == P.PNGF_ETIMEOUT
    assert int(ctx.counters.cpu()[6]) == P.PNGF_ETIMEOUT
    # the hold is one-shot; the latched status was cleared by the sync
    ctx.set_wait_limit(0, hold_cta=-1)
    ctx.restore()
    res = ctx.dbs_sweep(g["spec"]["n_sweeps"])
    assert _seq(res["trace"]) == [tuple(a[:3]) for a in g["accepted"]]
    o, f = ctx.eval_ports()
    want = np.array([complex(*z) for z in g["final_o"]])
    assert np.max(np.abs(o - want)) <= 1e-6 * np.max(np.abs(want))
    ctx.close()


def test_wait_limit_arguments_are_checked(P, fdfd64):
    ctx = P.DbsContext(fdfd64)
    for bad in [(3, -1), (31, -1), (0, -2), (0, 1 << 20)]:
        with pytest.raises(P.PngfError):
            ctx.set_wait_limit(*bad)
    ctx.close()


def test_fp64_checkpoint_resumes_bit_for_bit(P, fdfd64):
    order = W.shuffled_order(fdfd64.n_d, 6, seed=5)
    b0 = W.random_design(fdfd64.n_d, 2)
    kw = dict(tau=1e-9, refresh_k=16)
    whole = P.DbsContext(fdfd64, **kw)
    whole.factor(b0)
    ra = whole.dbs_sweep(6, order=order)
    o_a, f_a = whole.eval_ports()
    first = P.DbsContext(fdfd64, **kw)
    first.factor(b0)
    r1 = first.dbs_sweep(1, order=order[:1])
    ck = first.checkpoint()
    first.close()
    assert 0 <= ck["since_refresh"] < 16
    # a fresh context of the same inputs, factored at an unrelated design, takes the checkpoint
    second = P.DbsContext(fdfd64, **kw)
    second.factor(W.random_design(fdfd64.n_d, 99))
    second.set_state(ck)
    assert np.array_equal(second.design(), ck["b"])
    r2 = second.dbs_sweep(5, order=order[1:])
    o_b, f_b = second.eval_ports()
    resumed = _seq(r1["trace"]) + [(s + 1, t, k) for s, t, k in _seq(r2["trace"])]
    assert resumed == _seq(ra["trace"])
    assert np.array_equal(np.concatenate([r1["trace_f"], r2["trace_f"]]), ra["trace_f"])
    assert np.array_equal(o_a, o_b) and f_a == f_b
    assert np.array_equal(whole.design(), second.design())
    whole.close()
    second.close()


def test_mixed_checkpoint_resumes(P, fdfd64):
    g = _golden("fdfd64_first_raster")
    b0 = W.random_design(fdfd64.n_d, g["spec"]["seed"])
    kw = dict(tau=g["tau"], refresh_k=16, delay_r=8, precision=P.PNGF_MIXED, tensor_fold=1)
    first = P.DbsContext(fdfd64, **kw)
    first.factor(b0)
    r1 = first.dbs_sweep(1)
    ck = first.checkpoint()
    first.close()
    second = P.DbsContext(fdfd64, **kw)
    second.factor(ck["b"])  # mixed: factored at the checkpoint's design
    second.set_state(ck)
    r2 = second.dbs_sweep(g["spec"]["n_sweeps"] - 1)
    resumed = _seq(r1["trace"]) + [(s + 1, t, k) for s, t, k in _seq(r2["trace"])]
    assert resumed == [tuple(a[:3]) for a in g["accepted"]]
    o, _ = second.eval_ports()
    S = (o - fdfd64.s_off) * fdfd64.s_scale
    want = np.array([complex(*z) for z in g["final_o"]])
    S_want = (want - fdfd64.s_off) * fdfd64.s_scale
    assert np.max(np.abs(S - S_want) / np.maximum(np.abs(S_want), 1e-3)) < 1e-4
    # a mixed import takes neither b nor W (rejected before anything is read)
    import torch
    buf = torch.zeros(4 * fdfd64.n_d, dtype=torch.complex128, device="cuda")
    with pytest.raises(P.PngfError):
        P.pngf_set_state(second.ctx, buf.data_ptr(), None, buf.data_ptr(), buf.data_ptr(), buf.data_ptr(),
                         buf.data_ptr(), 0)
    second.close()


def test_batch_call_captured_in_cuda_graph(P, fdfd64):
    import torch

    dev = torch.device("cuda")
    s = torch.cuda.Stream(dev)
    subs = [fdfd64, fdfd64.sub_case(np.arange(0, 100, 2)), fdfd64.sub_case(np.arange(10, 74))]
    ctxs = []
    with torch.cuda.stream(s):
        for i, c in enumerate(subs * 2):
            cx = P.DbsContext(c, tau=1e-9, refresh_k=16, stream=s)
            cx.factor(W.random_design(c.n_d, i))
            cx.snapshot()
            ctxs.append(cx)
        cap = 6 * 100
        traces = [torch.zeros((cap, 4), dtype=torch.int32, device=dev) for _ in ctxs]
        trf = [torch.zeros(cap, dtype=torch.float64, device=dev) for _ in ctxs]
        cnt = torch.zeros((len(ctxs), 8), dtype=torch.int64, device=dev)
        ws_bytes = P.pngf_batch_workspace_size(len(ctxs))
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)

        def call():
            for cx in ctxs:
                P.pngf_restore(cx.ctx)
            P.pngf_dbs_sweep_batch([cx.ctx for cx in ctxs], 6, None, [t.data_ptr() for t in traces],
                                   [t.data_ptr() for t in trf], cap, cnt.data_ptr(), ws.data_ptr(), ws_bytes)

        call()
        s.synchronize()
    for cx in ctxs:
        assert cx.sync() == P.PNGF_OK
    eager = ([t.clone() for t in traces], [t.clone() for t in trf], cnt.clone(),
             [cx.eval_ports() for cx in ctxs])
    for t in traces:
        t.zero_()
    cnt.zero_()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        call()
    for _ in range(2):
        graph.replay()
        torch.cuda.synchronize()
        for cx in ctxs:
            assert cx.sync() == P.PNGF_OK
        assert torch.equal(cnt, eager[2])
        for a, b in zip(traces, eager[0]):
            assert torch.equal(a, b)
        for a, b in zip(trf, eager[1]):
            assert torch.equal(a, b)
        for cx, (o, f) in zip(ctxs, eager[3]):
            o2, f2 = cx.eval_ports()
            assert np.array_equal(o, o2) and f == f2
    for cx in ctxs:
        cx.close()


def test_mixed_accuracy_guard_stops_a_broken_state(P, fdfd64):
    """A mixed search whose maintained field no longer solves the system (here a
    checkpoint imported with e scaled by 1.5, a host-side stand-in for an FP32
    inverse that lost accuracy on an ill-conditioned system) stops at its next
    refresh with PNGF_EACCURACY instead of searching on a wrong state."""
    ctx = P.DbsContext(fdfd64, precision=P.PNGF_MIXED, tau=1e-9, delay_r=8, refresh_k=16, tensor_fold=1)
    ctx.factor(W.random_design(fdfd64.n_d, 0))
    ck = ctx.checkpoint()
    ck["e"] = ck["e"] * 1.5
    ck["since_refresh"] = 0
    ctx.set_state(ck)
    ctx.dbs_sweep(3, sync=False)
    assert ctx.sync() == P.PNGF_EACCURACY
    c = ctx.counters.cpu().numpy()
    assert c[6] == P.PNGF_EACCURACY and c[0] == 16  # stopped at the first refresh
    # the same context with a sound state searches normally
    ctx.factor(W.random_design(fdfd64.n_d, 0))
    g = _golden("fdfd64_first_raster")
    res = ctx.dbs_sweep(g["spec"]["n_sweeps"])
    assert _seq(res["trace"]) == [tuple(a[:3]) for a in g["accepted"]]
    ctx.close()
