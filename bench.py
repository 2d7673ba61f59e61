"""Benchmark of the PNGF direct-binary-search hot path on GB300.

One step = restore the factored start state (device copies inside the
workspace) + one complete DBS run on the device (first improvement, raster
order, until a sweep keeps no flip or ``--sweeps`` sweeps ran).  The metric is
attempted pixel flips per second in sequential DBS semantics (the paper's
Table 1 counting: every visited flip is one evaluation).  The factorisation of
M is timed separately (``factor_ms``), as the paper reports the initial
inversion apart from the optimisation time (Table 1).

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU FP64 oracle
(every candidate re-solved with LAPACK) on the same workload instead.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DBS pixel-flip evals/sec at N_d=4096, mixed vs FP64 at 1e-4 S-param err"
UNIT = "evals/s"
WORKLOAD = "fdfd256_nd4096"  # 256^2 FDFD, 16-cell PML, eps=2.2 slab, 64x64 design {1,10}, 2 ports


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--delay-r", type=int, default=64)
    ap.add_argument("--tensor-fold", type=int, default=1, choices=[0, 1],
                    help="mixed path: fold the delayed set with tcgen05 (1) or FP32 CUDA cores (0)")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--sweeps", type=int, default=10)
    ap.add_argument("--refresh-k", type=int, default=64)
    ap.add_argument("--tau", type=float, default=1e-9)
    ap.add_argument("--cpu-sample-evals", type=int, default=16)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def case_name(workload: str) -> str:
    return {"fdfd64_nd100": "fdfd64", "fdfd128_metal_nd1024": "fdfd128_metal",
            "fdfd256_nd4096": "fdfd256"}.get(workload, workload)


# ---------------------------------------------------------------- distributed plumbing
class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None

    def init(self, torch, backend="nccl"):
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, torch, x: float, device) -> float:
        if not self.pg:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=device)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, torch, x: float, device) -> float:
        if not self.pg:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=device)
        self.pg.all_reduce(t)
        return float(t.item())


# ---------------------------------------------------------------- clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = f"/tmp/pngf_clocks_{os.getpid()}.csv"

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except Exception:
        return {}


def fp64_peak_gflops(stream_handle) -> float:
    from paper_2501_18054_gb300 import build as B
    lib = ctypes.CDLL(B.build()["libpngf_peaks.so"])
    out = ctypes.c_double(0.0)
    rc = lib.pngf_peak_fp64_gflops(ctypes.byref(out), ctypes.c_int(3), ctypes.c_void_p(stream_handle))
    return float(out.value) if rc == 0 else float("nan")


# ---------------------------------------------------------------- CPU oracle timing
def time_oracle(case, b0, n_evals: int):
    import oracle as O
    p = O.Problem.from_case(case)
    t0 = time.perf_counter()
    res = O.dbs(p, b0, np.arange(case.n_d, dtype=np.int32)[None, :], tau=1e-9, max_evals=n_evals)
    dt = time.perf_counter() - t0
    return res.n_evals / dt, res.n_evals, dt


def blas_threads() -> int:
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(v):
            return int(os.environ[v])
    return os.cpu_count() or 1


def run_reference(args):
    dist = Dist()
    if dist.rank != 0:
        return 0
    from paper_2501_18054_gb300 import workloads as Wl
    case = Wl.get_case(case_name(args.workload))
    b0 = Wl.random_design(case.n_d, 0)
    per_step = max(1, min(args.cpu_sample_evals // 4, 8))
    for _ in range(args.warmup):
        time_oracle(case, b0, per_step)
    t0 = time.perf_counter()
    n = 0
    for _ in range(args.steps):
        _, m, _ = time_oracle(case, b0, per_step)
        n += m
    dt = time.perf_counter() - t0
    value = n / dt
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
                ms_per_step=dt * 1e3 / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic", impl="reference",
                config={"workload": args.workload, "n_d": case.n_d, "n_o": case.n_o,
                        "sample": f"first {per_step} attempted flips of the raster DBS run per step"},
                cpu_baseline={"value": value, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
                              "sample": f"{per_step} candidate re-solves (LAPACK zgesv, n={case.n_d}) per step"},
                e2e={"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0})
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- batched workload
BATCH_WORKLOAD = "batch256_fdfd128_metal"  # 256 runs, N_d in {256, 576, 1024} sub-blocks of one G


def batch_cases(Wl):
    """The batched workload: random starts b = 0..255 on the 128^2 lossy-metal device.

    Run b uses the principal sub-block [256, 576, 1024][b % 3] of the 32 x 32
    design region (16 x 16 at offset (8, 8), 24 x 24 at (4, 4), the whole
    region), seed b; the three sub-block Green functions are shared.
    """
    big = Wl.get_case("fdfd128_metal")

    def block(x0, side):
        return np.array([(x0 + i) * 32 + (x0 + j) for i in range(side) for j in range(side)])

    subs = [big.sub_case(block(8, 16), "metal_sub256"), big.sub_case(block(4, 24), "metal_sub576"), big]
    return [(subs[b % 3], b) for b in range(256)]


def bench_batch(args, torch, dist, dev, P, Wl):
    runs = batch_cases(Wl)
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        shared = {}
        ctxs = []
        t_f0 = time.perf_counter()
        for case, seed in runs:
            if case.name not in shared:
                c0 = P.DbsContext(case, precision=P.PNGF_FP64, tau=args.tau, refresh_k=args.refresh_k,
                                  device=str(dev), stream=stream)
                shared[case.name] = (c0.G, c0.God, c0.cd, c0.co, c0.dv)
                ctx = c0
            else:
                ctx = P.DbsContext(case, precision=P.PNGF_FP64, tau=args.tau, refresh_k=args.refresh_k,
                                   device=str(dev), stream=stream, inputs_on_device=shared[case.name])
            ctx.factor(Wl.random_design(case.n_d, seed + 1000 * dist.rank))
            ctxs.append(ctx)
        stream.synchronize()
        factor_s = time.perf_counter() - t_f0
        for c in ctxs:
            if c.sync() != 0:
                raise RuntimeError("factor failed")
            c.snapshot()
        batch = P.DbsBatch(ctxs)
        trace_cap = args.sweeps * 1024
        traces = [torch.zeros((trace_cap, 4), dtype=torch.int32, device=dev) for _ in ctxs]
        counters = batch.counters

        def step():
            for c in ctxs:
                P.pngf_restore(c.ctx)
            P.pngf_dbs_sweep_batch([c.ctx for c in ctxs], args.sweeps, None, [t.data_ptr() for t in traces], None,
                                   trace_cap, counters.data_ptr(), batch.ws.data_ptr(), batch.ws_bytes)

        for _ in range(max(args.warmup, 1)):
            step()
        stream.synchronize()
        cnt = counters.cpu().numpy().copy()
        evals = int(cnt[:, 1].sum())
        peak_fp64 = fp64_peak_gflops(stream.cuda_stream)
        dist.barrier()
        torch.cuda.synchronize(dev)
        clocks = Clocks(dist.local)
        clocks.start()
        time.sleep(0.3)
        kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for i in range(args.steps):
            for c in ctxs:
                P.pngf_restore(c.ctx)
            kev[i][0].record(stream)
            P.pngf_dbs_sweep_batch([c.ctx for c in ctxs], args.sweeps, None, [t.data_ptr() for t in traces], None,
                                   trace_cap, counters.data_ptr(), batch.ws.data_ptr(), batch.ws_bytes)
            kev[i][1].record(stream)
        t1.record(stream)
        stream.synchronize()
        clk = clocks.stop()
        dist.barrier()
        for c in ctxs:
            if c.sync() != 0:
                raise RuntimeError("batched steps failed")
        cnt2 = counters.cpu().numpy()
        assert int(cnt2[:, 1].sum()) == evals
        ms = t0.elapsed_time(t1)
        ms_max = dist.max(torch, ms, dev)
        total = dist.sum(torch, float(evals * args.steps), dev)
        value = total / (ms_max / 1e3)
        k_avg = sum(a.elapsed_time(b) for a, b in kev) / args.steps
        # algorithmic FP64 work of the batched kernel per launch: the rank-1 update of
        # the upper triangle per kept flip (8 flop per element) plus per refresh the
        # FP64 residual G x over (1 + n_o) vectors (8 flop per complex multiply-add)
        flops = 0.0
        for (case, _), row in zip(runs, cnt2):
            n = case.n_d
            flops += row[0] * 8.0 * n * (n + 1) / 2 + row[4] * 8.0 * n * n * (1 + case.n_o)
        gf = flops / (k_avg / 1e3) / 1e9
        roofline = {"bound": "alu", "achieved": gf / 1e3, "peak": peak_fp64 / 1e3, "unit": "TFLOP/s",
                    "frac": gf / peak_fp64, "traffic": None, "kernel": "dbs_batch_kernel",
                    "peak_source": "FP64 FMA pipe, measured in this run by libpngf_peaks"}
    if dist.rank == 0:
        line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=dist.world, steps=args.steps, warmup=args.warmup,
                    ms_per_step=ms_max / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                    dtype="f64", data="synthetic",
                    config={"workload": BATCH_WORKLOAD, "runs": len(runs), "n_d": "256/576/1024 (b mod 3)",
                            "precision": "fp64", "mode": "first-improvement, raster order",
                            "max_sweeps": args.sweeps, "refresh_k": args.refresh_k, "tau": args.tau,
                            "step": "restore every run's factored start + one batched launch to convergence",
                            "l2": "inputs larger than L2 (W of all runs ~%.1f GB)" % (
                                sum(c.n_d ** 2 for c, _ in runs) * 16 / 1e9)},
                    roofline=roofline, cpu_baseline=None, e2e=None, clocks=clk, gpu_launches=args.steps,
                    evals_per_step=evals, accepts_per_step=int(cnt2[:, 0].sum()),
                    converged_runs=int(cnt2[:, 3].sum()), kernel_ms_avg=k_avg, factor_s_all_runs=factor_s,
                    fp64_peak_gflops=peak_fp64)
        print(json.dumps(line))
    for c in ctxs:
        c.close()
    return 0


# ---------------------------------------------------------------- GPU arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch

    dist = Dist()
    torch.cuda.set_device(dist.local)
    dev = torch.device("cuda", dist.local)
    dist.init(torch)
    from paper_2501_18054_gb300 import build as B
    if dist.rank == 0:
        B.build()
    dist.barrier()
    B.build()
    from paper_2501_18054_gb300 import pngf as P
    from paper_2501_18054_gb300 import workloads as Wl

    if args.workload == BATCH_WORKLOAD:
        return bench_batch(args, torch, dist, dev, P, Wl)
    case = Wl.get_case(case_name(args.workload))
    n, n_o = case.n_d, case.n_o
    prec = P.PNGF_MIXED if args.precision == "mixed" else P.PNGF_FP64
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        ctx = P.DbsContext(case, precision=prec, tau=args.tau, refresh_k=args.refresh_k, delay_r=args.delay_r,
                           device=str(dev), stream=stream, tensor_fold=args.tensor_fold)
        b0 = Wl.random_design(n, seed=dist.rank)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.factor(b0)
        e1.record(stream)
        stream.synchronize()
        factor_ms = e0.elapsed_time(e1)
        st = ctx.sync()
        if st != 0:
            raise P.PngfError(st, "pngf_factor")
        ctx.snapshot()
        trace_cap = args.sweeps * n
        trace = torch.zeros((trace_cap, 4), dtype=torch.int32, device=dev)
        trace_f = torch.zeros(trace_cap, dtype=torch.float64, device=dev)
        counters = torch.zeros(8, dtype=torch.int64, device=dev)
        kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]

        def step(i=None, order_ptr=None):
            P.pngf_restore(ctx.ctx)
            if i is not None:
                kev[i][0].record(stream)
            P.pngf_dbs_sweep(ctx.ctx, args.sweeps, order_ptr, trace.data_ptr(), trace_f.data_ptr(), trace_cap,
                             counters.data_ptr())
            if i is not None:
                kev[i][1].record(stream)

        for _ in range(max(args.warmup, 1)):
            step()
        stream.synchronize()
        st = ctx.sync()
        if st not in (0,):
            raise P.PngfError(st, "warm-up")
        c = counters.cpu().numpy().copy()
        evals_per_step, acc_per_step, sweeps_per_step = int(c[1]), int(c[0]), int(c[2])
        peak_fp64 = fp64_peak_gflops(stream.cuda_stream)
        # ---- timed region (device time, CUDA events on the launching stream)
        dist.barrier()
        torch.cuda.synchronize(dev)
        clocks = Clocks(dist.local)
        clocks.start()
        time.sleep(0.3)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for i in range(args.steps):
            step(i)
        t1.record(stream)
        stream.synchronize()
        torch.cuda.synchronize(dev)
        clk = clocks.stop()
        dist.barrier()
        st = ctx.sync()
        if st != 0:
            raise P.PngfError(st, "timed steps")
        c2 = counters.cpu().numpy()
        assert int(c2[1]) == evals_per_step, "steps are not identical runs"
        cyc = ctx.phase_cycles()
        mhz = clk.get("sm_mhz") or 2070.0
        phase_names = ["score", "wait_after_score", "select_pivot_gather", "wait_or_flush",
                       "update", "refresh", "sweep_setup", "kernel_total", "refresh_x", "refresh_residual",
                       "refresh_correct", "refresh_ports", "publish", "update_delayed_sum",
                       "unused14", "unused15"]
        phase_ms = {nm: float(cv) / (mhz * 1e3) for nm, cv in zip(phase_names, cyc)}
        ms = t0.elapsed_time(t1)
        ms_max = dist.max(torch, ms, dev)
        total_evals = dist.sum(torch, float(evals_per_step * args.steps), dev)
        value = total_evals / (ms_max / 1e3)
        kms = [a.elapsed_time(b) for a, b in kev]
        k_avg = sum(kms) / len(kms)
        peaks = measured_peaks()
        hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
        tri = n * (n + 1) / 2
        if prec == P.PNGF_FP64:
            # dominant kernel: the persistent FP64 DBS sweep.  Algorithmic work per
            # launch: the rank-1 update of the upper triangle of W per kept flip,
            # 4 DFMA = 8 flop per complex element (32 bytes of W read + written).
            flops = acc_per_step * 8.0 * tri
            bytes_w = acc_per_step * 32.0 * tri
            achieved_gflops = flops / (k_avg / 1e3) / 1e9
            roofline = {"bound": "alu", "achieved": achieved_gflops / 1e3, "peak": peak_fp64 / 1e3,
                        "unit": "TFLOP/s", "frac": achieved_gflops / peak_fp64, "traffic": None,
                        "kernel": "dbs_fp64_kernel",
                        "peak_source": "FP64 FMA pipe, measured in this run by libpngf_peaks "
                                       "(152 SMs x 2 DFMA/clk x 2 flop x clock)",
                        "hbm_view": {"achieved_gbs": bytes_w / (k_avg / 1e3) / 1e9, "peak_gbs": hbm_peak,
                                     "frac": bytes_w / (k_avg / 1e3) / 1e9 / hbm_peak,
                                     "peak_source": "MEASURED_PEAKS.json hbm_gbs"}}
        else:
            # dominant kernel: the persistent mixed DBS sweep.  Algorithmic HBM bytes per
            # launch: per flush the upper triangle of the two FP32 planes read + written
            # (16 B per element), per refresh one read of G (16 B) and of the FP32
            # upper triangle (8 B), per kept flip one column of the FP32 planes (8 B x n),
            # per evaluation (3 + n_o) x 16 B of FP64 state.
            n_flush, n_ref = int(c2[5]), int(c2[4])
            bytes_alg = (n_flush * 16.0 * tri + n_ref * (16.0 * n * n + 8.0 * tri) + acc_per_step * 8.0 * n
                         + evals_per_step * (3 + n_o) * 16.0)
            gbs = bytes_alg / (k_avg / 1e3) / 1e9
            roofline = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                        "traffic": None, "kernel": "dbs_mixed_kernel",
                        "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst copy)",
                        "note": "one kept flip at a time: the single-run search is latency-bound "
                                "(grid barrier + selection per kept flip); see phase_ms_cta0"}
        # ---- end to end through the C ABI with host buffers
        e2e = None
        if not args.no_e2e:
            order_h = torch.from_numpy(np.tile(np.arange(n, dtype=np.int32), (args.sweeps, 1))).pin_memory()
            order_d = torch.empty_like(order_h, device=dev)
            trace_h = torch.empty((trace_cap, 4), dtype=torch.int32).pin_memory()
            trace_fh = torch.empty(trace_cap, dtype=torch.float64).pin_memory()
            cnt_h = torch.empty(8, dtype=torch.int64).pin_memory()
            h2d = order_h.numel() * 4
            d2h = trace_h.numel() * 4 + trace_fh.numel() * 8 + cnt_h.numel() * 8 + 16 * n_o + 8
            for rep in range(2):
                dist.barrier()
                torch.cuda.synchronize(dev)
                w0 = time.perf_counter()
                for i in range(args.steps):
                    order_d.copy_(order_h, non_blocking=True)
                    step(None, order_d.data_ptr())
                    trace_h.copy_(trace, non_blocking=True)
                    trace_fh.copy_(trace_f, non_blocking=True)
                    cnt_h.copy_(counters, non_blocking=True)
                    o_host, f_host = ctx.eval_ports()  # synchronizes: the step's result on the host
                w1 = time.perf_counter()
            assert int(cnt_h[1]) == evals_per_step
            e2e_s = dist.max(torch, w1 - w0, dev)
            e2e = {"value": total_evals / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                   "d2h_bytes_per_step": int(d2h)}
        # ---- the same run on the FP64 path (same GPU, same start) for the speedup and
        #      the S-parameter error of the mixed path
        compare = None
        restore_and_run = step
        restore_and_run()
        stream.synchronize()
        o_main, f_main = ctx.eval_ports()
        b_main = ctx.design()
        trace_main = trace[:min(acc_per_step, trace_cap), 2].cpu().numpy().copy()
        if prec == P.PNGF_MIXED and not args.no_fp64_compare:
            ref = P.DbsContext(case, precision=P.PNGF_FP64, tau=args.tau, refresh_k=args.refresh_k, device=str(dev),
                               stream=stream, inputs_on_device=(ctx.G, ctx.God, ctx.cd, ctx.co, ctx.dv))
            ref.factor(b0)
            ref.snapshot()
            cnt64 = torch.zeros(8, dtype=torch.int64, device=dev)
            tr64 = torch.zeros((trace_cap, 4), dtype=torch.int32, device=dev)

            def step64():
                P.pngf_restore(ref.ctx)
                P.pngf_dbs_sweep(ref.ctx, args.sweeps, None, tr64.data_ptr(), None, trace_cap, cnt64.data_ptr())

            step64()
            stream.synchronize()
            r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 2
            r0.record(stream)
            for _ in range(reps):
                step64()
            r1.record(stream)
            stream.synchronize()
            if ref.sync() != 0:
                raise RuntimeError("FP64 comparison run failed")
            c64 = cnt64.cpu().numpy()
            ms64 = r0.elapsed_time(r1) / reps
            o64, f64 = ref.eval_ports()
            b64 = ref.design()
            k64 = tr64[:min(int(c64[0]), trace_cap), 2].cpu().numpy()
            same = bool(np.array_equal(b64, b_main))
            prefix = next((i for i, (x, y) in enumerate(zip(k64, trace_main)) if x != y), min(len(k64), len(trace_main)))
            S_main = (o_main - case.s_off) * case.s_scale
            S_64 = (o64 - case.s_off) * case.s_scale
            compare = {"fp64_evals_per_s": float(c64[1]) / (ms64 / 1e3), "fp64_ms_per_step": ms64,
                       "speedup_vs_fp64": (float(c64[1]) / (ms64 / 1e3)) and value / (float(c64[1]) / (ms64 / 1e3)),
                       "same_final_design": same, "identical_accept_prefix": int(prefix),
                       "accepts_fp64": int(c64[0]), "accepts_mixed": int(acc_per_step)}
            if same:
                compare["s_param_max_rel_err_vs_fp64"] = float(
                    np.max(np.abs(S_main - S_64) / np.maximum(np.abs(S_64), 1e-3)))
            ref.close()
        if dist.rank == 0:
            import oracle as O
            ev = O.evaluate(O.Problem.from_case(case), b_main)
            S_exact = (ev.o - case.s_off) * case.s_scale
            S_main = (o_main - case.s_off) * case.s_scale
            compare = dict(compare or {})
            compare["s_param_max_rel_err_vs_oracle"] = float(
                np.max(np.abs(S_main - S_exact) / np.maximum(np.abs(S_exact), 1e-3)))
            compare["s_param_err_note"] = "final design of the timed run, exact S from the CPU FP64 oracle"
        cpu = None
        if dist.rank == 0 and not args.no_cpu_baseline:
            v, m, dt = time_oracle(case, b0, args.cpu_sample_evals)
            cpu = {"value": v, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
                   "sample": f"first {m} attempted flips of the same raster DBS run, each re-solved with "
                             f"LAPACK zgesv at n={n} ({dt:.1f} s)"}
    if dist.rank == 0:
        line = dict(
            metric=METRIC, value=value, unit=UNIT, n_gpus=dist.world, steps=args.steps, warmup=args.warmup,
            ms_per_step=ms_max / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
            dtype="f64" if prec == P.PNGF_FP64 else "f32+f64", data="synthetic",
            config={"workload": args.workload, "n_d": n, "n_o": n_o, "precision": args.precision,
                    "mode": "first-improvement, raster order", "max_sweeps": args.sweeps,
                    "refresh_k": args.refresh_k, "tau": args.tau,
                    "delay_r": args.delay_r if prec == P.PNGF_MIXED else None,
                    "fold": ("tcgen05 3xTF32" if args.tensor_fold else "FP32 CUDA cores")
                    if prec == P.PNGF_MIXED else None,
                    "step": "restore factored start state + DBS run to convergence",
                    "l2": "inputs larger than L2 (W = %.0f MB complex128)" % (n * n * 16 / 1e6),
                    "replicas": "one independent run per GPU (seed = rank)"},
            roofline=roofline, cpu_baseline=cpu, e2e=e2e, clocks=clk, gpu_launches=args.steps,
            evals_per_step=evals_per_step, accepts_per_step=acc_per_step, sweeps_per_step=sweeps_per_step,
            accepts_per_s=acc_per_step * args.steps / (ms_max / 1e3),
            sweeps_per_s=sweeps_per_step * args.steps / (ms_max / 1e3),
            kernel_ms_avg=k_avg, factor_ms=factor_ms, fp64_peak_gflops=peak_fp64, phase_ms_cta0=phase_ms,
            mixed_vs_fp64=compare)
        print(json.dumps(line))
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
