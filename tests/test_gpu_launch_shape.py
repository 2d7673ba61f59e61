"""The headline workload (fdfd256, N_d = 4096, mixed precision, R = 64, a
refresh every 64 kept flips) at the launch shapes the bench uses: several
independent runs side by side on one GPU, each a cooperative launch on its own
stream with an equal share of the SMs (4 runs of 38 CTAs, 108 pixels per CTA;
8 runs of 19 CTAs, 216 pixels per CTA).  Every run must end on the FP64 path's
final design from the same start, with S-parameters within the mixed path's
1e-4 of the oracle's for that design.
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


@pytest.fixture(scope="module")
def fdfd256():
    return W.get_case("fdfd256")


def _runs(P, case, runs, precision, inputs=None):
    import torch

    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    ctas = nsm // runs
    streams = [torch.cuda.Stream() for _ in range(runs)]
    ctxs = []
    for i, s in enumerate(streams):
        kw = dict(precision=precision, tau=1e-9, refresh_k=64, n_ctas=ctas, stream=s)
        if precision == P.PNGF_MIXED:
            kw.update(delay_r=64, tensor_fold=1)
        if inputs is not None:
            kw["inputs_on_device"] = inputs
        cx = P.DbsContext(case, **kw)
        inputs = inputs or (cx.G, cx.God, cx.cd, cx.co, cx.dv)
        cx.factor(W.random_design(case.n_d, i))
        ctxs.append(cx)
    torch.cuda.synchronize()
    for cx in ctxs:  # launched side by side: each on its own stream
        cx.dbs_sweep(10, sync=False)
    torch.cuda.synchronize()
    for cx in ctxs:
        assert cx.sync() == P.PNGF_OK
    return ctxs, inputs


@pytest.mark.parametrize("runs", [4, 8])
def test_concurrent_runs_at_the_bench_shape(P, fdfd256, runs):
    case = fdfd256
    mixed, inputs = _runs(P, case, runs, P.PNGF_MIXED)
    ref, _ = _runs(P, case, runs, P.PNGF_FP64, inputs)
    p = O.Problem.from_case(case)
    for i, (cm, cf) in enumerate(zip(mixed, ref)):
        assert int(cm.counters.cpu()[0]) > 100
        b = cm.design()
        assert np.array_equal(b, cf.design()), f"run {i}: final design differs from the FP64 path's"
        o, _ = cm.eval_ports()
        ev = O.evaluate(p, b)
        S = (o - case.s_off) * case.s_scale
        S_ex = (ev.o - case.s_off) * case.s_scale
        assert np.max(np.abs(S - S_ex) / np.maximum(np.abs(S_ex), 1e-3)) < 1e-4
    for cx in mixed + ref:
        cx.close()
