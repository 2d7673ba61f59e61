"""Benchmark of the PNGF direct-binary-search hot path on GB300.

One step = for each of ``--runs`` independent random starts (default 4):
restore the factored start state (device copies inside the workspace) + one
complete DBS run on the device (first improvement, raster order, until a
sweep keeps no flip or ``--sweeps`` sweeps ran); the runs' persistent launches
execute side by side, each on its own stream and share of the SMs.  The metric is
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

# DRAM traffic of the search kernel from one ncu capture of that kernel on this workload
# (one launch = one full run, seed 0): measured read + write bytes over the algorithmic bytes of
# that launch.  A step's traffic is this ratio times the step's algorithmic bytes, reported only
# while the kernel code is the captured one (fingerprint of the sources without comments), else null.
TRAFFIC_CAPTURE = {"kernel": "dbs_mixed_kernel", "workload": "fdfd256_nd4096",
                   "measured_bytes": 2.670050e9 + 0.985426e9, "algorithmic_bytes": 4509239696.0,
                   "sources_sha256": "09b40a5bcb8a90e27b313f1f144accac2e1c45406aac6979374347a0fd716312"}


def _code_only(src: str) -> str:
    """C/C++ source without its comments and blank space, so that an edit of the
    comments alone leaves the fingerprint of the code unchanged; string and
    character literals are kept as they are."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            i = src.find("\n", i)
            i = n if i < 0 else i
        elif src.startswith("/*", i):
            i = src.find("*/", i + 2)
            i = n if i < 0 else i + 2
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


# the sources the mixed search kernel and its launch are built from
MIXED_KERNEL_SOURCES = ("sweep_mixed.cu", "flush_tc.cuh", "refresh_df.cuh", "dd.cuh", "sweep_common.cuh",
                        "mixed_common.cuh", "pngf_internal.cuh", "api.cu")


def sources_fingerprint() -> str:
    """sha256 over the code (comments and blank space removed) of the mixed
    search kernel's sources and the C ABI header."""
    import hashlib
    files = [os.path.join(ROOT, "paper_2501_18054_gb300", "csrc", f) for f in MIXED_KERNEL_SOURCES]
    files.append(os.path.join(ROOT, "include", "pngf.h"))
    h = hashlib.sha256()
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()


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
    ap.add_argument("--runs", type=int, default=4,
                    help="independent runs side by side on their own streams (concurrent slots)")
    ap.add_argument("--runs-per-slot", type=int, default=4,
                    help="mixed/FP64 headline: runs queued one after another on each slot's stream; a step "
                         "is runs x runs-per-slot independent searches")
    # kept flips between refreshes of the mixed path (a multiple of --delay-r); the headline
    # configuration refreshes every 64 kept flips
    ap.add_argument("--refresh-k", type=int, default=64)
    ap.add_argument("--tau", type=float, default=1e-9)
    ap.add_argument("--cpu-sample-evals", type=int, default=16)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-one-core", action="store_true",
                    help="also time the oracle with one BLAS thread (two solves, ~1 min at N_d = 4096)")
    ap.add_argument("--cpu-kept-flips", type=int, default=300,
                    help="kept flips of the numpy Sherman-Morrison baseline's sample")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--ctas-per-run", type=int, default=0,
                    help="CTAs of each run's cooperative launch (0: the SMs divided among the runs)")
    ap.add_argument("--hankel-sweeps", type=int, default=2,
                    help="hankel128_nd16384: sweeps per run (the third drives the lossless design into a "
                         "high-Q resonance where the FP32 inverse of the mixed path stops with PNGF_EACCURACY)")
    ap.add_argument("--side-runs", type=int, default=8,
                    help="pec/tiles/multifreq workloads: independent searches side by side (nsm / runs CTAs each)")
    ap.add_argument("--autotune", type=int, default=1, choices=[0, 1],
                    help="mixed path: choose runs per GPU, delay R and fold engine from timed trials first")
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


def replica_seeds(rank: int, runs: int) -> list:
    """Seeds of one rank's independent runs: disjoint across ranks (rank * runs + i)."""
    return [rank * runs + i for i in range(runs)]


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


def time_paper_algorithm(case, b0, n_kept: int, sweeps: int = 10):
    """The paper's own CPU algorithm written plainly with numpy and the threaded
    BLAS (the counterpart of Table 1's "PNGF on BLAS/LAPACK"): factor once
    (LAPACK solve for W = M^-1 G and e, T = G_od (I + V W)), then first-improvement
    DBS in raster order where every candidate is scored in O(n_o) (Eq. 14, field
    form) and a kept flip updates W, T, e by rank 1 (Eq. 9, BLAS zgeru in place).
    Returns (evals/s, evaluations, kept flips, seconds of search, seconds of factor)
    over the first ``n_kept`` kept flips of the run."""
    import scipy.linalg as sla
    from scipy.linalg import blas
    n, G = case.n_d, case.G_dd
    dv, s_off, s_scale, w = case.dv, case.s_off, case.s_scale, case.obj_weights
    kind = int(case.obj_kind)

    def fobj(o):  # o: (n_o, m) port amplitudes -> objective per column
        a = np.abs((o - s_off[:, None]) * s_scale[:, None])
        return np.sum(w[:, None] * (a * a if kind == 0 else (1.0 - a) ** 2), axis=0)

    b = np.asarray(b0, dtype=np.uint8).copy()
    t0 = time.perf_counter()
    v = dv * b
    sol = sla.solve(np.eye(n, dtype=np.complex128) - G * v[None, :], np.concatenate([G, case.c_d[:, None]], 1))
    W = np.ascontiguousarray(sol[:, :n])
    e = sol[:, n].copy()
    T = case.G_od + (case.G_od * v[None, :]) @ W
    o = case.c_o + case.G_od @ (v * e)
    t_factor = time.perf_counter() - t0
    f = float(fobj(o[:, None])[0])
    evals = kept = 0
    t0 = time.perf_counter()
    for _ in range(sweeps):
        t, kept_in_sweep = 0, 0
        while t < n and kept < n_kept:
            delta = np.where(b[t:] == 1, -dv[t:], dv[t:])
            d = 1.0 - delta * np.diagonal(W)[t:]
            alpha = delta / d
            coef = alpha * e[t:]
            fn = fobj(o[:, None] + coef[None, :] * T[:, t:])
            gain = fn - f if kind == 0 else f - fn
            hit = np.flatnonzero(gain > 1e-9 * max(abs(f), 1e-30))
            if len(hit) == 0:
                evals += n - t
                t = n
                break
            q = int(hit[0])
            k = t + q
            evals += q + 1
            c = W[:, k].copy()
            Tk = T[:, k].copy()
            blas.zgeru(alpha[q], c, c, a=W.T, overwrite_a=1)  # W += alpha c c^T (W symmetric)
            T += alpha[q] * np.outer(Tk, c)
            e += coef[q] * c
            o = o + coef[q] * Tk
            f = float(fn[q])
            b[k] ^= 1
            kept += 1
            kept_in_sweep += 1
            t = k + 1
        if kept >= n_kept or kept_in_sweep == 0:
            break
    dt = time.perf_counter() - t0
    return evals / dt, evals, kept, dt, t_factor


def time_oracle_one_core(workload: str, n_evals: int):
    """The oracle timed in a child process limited to one BLAS thread."""
    code = ("import json, sys; sys.path.insert(0, %r); import bench, numpy as np; "
            "from paper_2501_18054_gb300 import workloads as Wl; "
            "c = Wl.get_case(bench.case_name(%r)); "
            "print(json.dumps(bench.time_oracle(c, Wl.random_design(c.n_d, 0), %d)))" % (ROOT, workload, n_evals))
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        v, m, dt = json.loads(r.stdout.strip().splitlines()[-1])
        return {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"first {m} attempted flips re-solved with one BLAS thread ({dt:.1f} s)"}
    except Exception as ex:  # a baseline, not the measurement: report why it is missing
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "error": str(ex)[:200]}


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
                            "step": "restore every run's factored start + one batched launch, up to %d sweeps "
                                    "or until a sweep keeps no flip" % args.sweeps,
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


def mixed_alg_bytes(c2, n, n_o) -> float:
    """Algorithmic HBM bytes of the mixed search's launches, from their counters
    (rows: runs; [0] kept flips, [1] evaluations, [4] refreshes, [5] folds,
    [7] active pixels summed over the refreshes): per fold the upper triangle of
    the two FP32 planes read + written (16 B per element); per refresh with m
    active pixels the m rows of G as FP32 pairs (16 B x m x n), the FP32 upper
    triangle (8 B) and its entries in the active rows above each column strip
    (8 B x m / n per element); per kept flip one column of the FP32 planes
    (8 B x n); per evaluation (3 + n_o) x 16 B of state."""
    c2 = np.atleast_2d(c2)
    tri = n * (n + 1) / 2
    n_flush, n_ref, sum_m = float(c2[:, 5].sum()), float(c2[:, 4].sum()), float(c2[:, 7].sum())
    return (n_flush * 16.0 * tri + 16.0 * n * sum_m + n_ref * 8.0 * tri + 8.0 * tri * sum_m / n
            + float(c2[:, 0].sum()) * 8.0 * n + float(c2[:, 1].sum()) * (3 + n_o) * 16.0)


# ---------------------------------------------------------------- the other paths, one run each
# name -> (what, case, extra): FP64-family searches and the gradient, each timed like the
# headline (restore + one complete search per step, CUDA events on the launching stream)
SIDE_WORKLOADS = {
    "pec_fdfd128_nd1024": "perfect-conductor pixels (Eq. 2) on the 128^2 slab device, 32x32 region, FP64",
    "tiles2x2_fdfd128_metal_nd1024": "2x2 tile flips (rank 4) on the 128^2 lossy-metal device, FP64",
    "multifreq3_fdfd128_metal_nd1024": "3 frequencies (wavelengths 19, 20, 21 cells) sharing the design, "
                                       "pixel flips, mean objective, FP64",
    "gradient_fdfd256_nd4096": "objective gradient at a random design of the 64x64 region (mixed context)",
    "hankel128_nd16384": "closed-form 2D Green function, 128x128 region (N_d = 16384), 4 ring ports, mixed "
                         "precision, one run on all SMs",
}


def bench_hankel(args, torch, dist, dev, P, Wl):
    """The largest region: one mixed run (R = 64, refresh every 64 kept flips), the
    final design's S-parameters checked against one oracle solve of that design."""
    import oracle as O
    case = Wl.get_case("hankel128")
    n, n_o = case.n_d, case.n_o
    stream = torch.cuda.Stream(dev)
    peaks = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    with torch.cuda.stream(stream):
        ctx = P.DbsContext(case, precision=P.PNGF_MIXED, tau=args.tau, refresh_k=args.refresh_k,
                           delay_r=args.delay_r, tensor_fold=args.tensor_fold, device=str(dev), stream=stream)
        b0 = Wl.random_design(n, 0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.factor(b0)
        e1.record(stream)
        stream.synchronize()
        factor_ms = e0.elapsed_time(e1)
        if ctx.sync() != 0:
            raise RuntimeError("hankel: factor failed")
        ctx.snapshot()
        cnt = torch.zeros(8, dtype=torch.int64, device=dev)

        sweeps = args.hankel_sweeps

        def step():
            P.pngf_restore(ctx.ctx)
            P.pngf_dbs_sweep(ctx.ctx, sweeps, None, None, None, 0, cnt.data_ptr())

        for _ in range(max(args.warmup, 1)):
            step()
        stream.synchronize()
        if ctx.sync() != 0:
            raise RuntimeError("hankel: warm-up failed")
        clocks = Clocks(dist.local)
        clocks.start()
        time.sleep(0.3)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            step()
        t1.record(stream)
        stream.synchronize()
        clk = clocks.stop()
    if ctx.sync() != 0:
        raise RuntimeError("hankel: timed steps failed")
    ms = t0.elapsed_time(t1) / args.steps
    c2 = cnt.cpu().numpy()
    value = float(c2[1]) / (ms / 1e3)
    bytes_alg = mixed_alg_bytes(c2, n, n_o)
    gbs = bytes_alg / (ms / 1e3) / 1e9
    o_gpu, _ = ctx.eval_ports()
    b_end = ctx.design()
    ts = time.perf_counter()
    ev = O.evaluate(O.Problem.from_case(case), b_end)
    oracle_s = time.perf_counter() - ts
    S_ex = (ev.o - case.s_off) * case.s_scale
    S_g = (o_gpu - case.s_off) * case.s_scale
    s_err = float(np.max(np.abs(S_g - S_ex) / np.maximum(np.abs(S_ex), 1e-3)))
    ctx.close()
    # the FP64 path on the same start and sweeps: its design, speed and the mixed path's speedup
    with torch.cuda.stream(stream):
        c64 = P.DbsContext(case, precision=P.PNGF_FP64, tau=args.tau, refresh_k=args.refresh_k, device=str(dev),
                           stream=stream, inputs_on_device=(ctx.G, ctx.God, ctx.cd, ctx.co, ctx.dv))
        c64.factor(b0)
        cnt64 = torch.zeros(8, dtype=torch.int64, device=dev)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        P.pngf_dbs_sweep(c64.ctx, sweeps, None, None, None, 0, cnt64.data_ptr())
        a1.record(stream)
        stream.synchronize()
    if c64.sync() != 0:
        raise RuntimeError("hankel: FP64 run failed")
    ev64 = float(cnt64.cpu().numpy()[1]) / (a0.elapsed_time(a1) / 1e3)
    same = bool(np.array_equal(c64.design(), b_end))
    c64.close()
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=dist.world, steps=args.steps, warmup=args.warmup,
                ms_per_step=ms, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32+f64",
                data="synthetic",
                config={"workload": "hankel128_nd16384", "what": SIDE_WORKLOADS["hankel128_nd16384"], "n_d": n,
                        "n_o": n_o, "runs": 1, "max_sweeps": sweeps, "refresh_k": args.refresh_k,
                        "delay_r": args.delay_r, "step": "restore the factored start + one search",
                        "note": "the configuration's 16 batched runs do not fit at once: each mixed context "
                                "holds ~20 GB (FP64 factor scratch included), and each FP64 factor takes "
                                "tens of seconds; one run is measured"},
                roofline={"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                          "traffic": None, "kernel": "dbs_mixed_kernel", "algorithmic_bytes_per_step": bytes_alg},
                accepts_per_step=int(c2[0]), evals_per_step=int(c2[1]), refreshes=int(c2[4]), folds=int(c2[5]),
                factor_ms=factor_ms, s_param_rel_err_vs_oracle=s_err, oracle_solve_s=oracle_s, clocks=clk,
                mixed_vs_fp64={"fp64_evals_per_s": ev64, "speedup_vs_fp64": value / ev64,
                               "same_final_design": same},
                gpu_launches=args.steps, cpu_baseline=None, e2e=None)
    if dist.rank == 0:
        print(json.dumps(line))
    return 0


def bench_side(args, torch, dist, dev, P, Wl):
    name = args.workload
    stream = torch.cuda.Stream(dev)
    peak_fp64 = fp64_peak_gflops(stream.cuda_stream)
    peaks = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    sweeps = args.sweeps
    ctxs, extra = [], {}
    with torch.cuda.stream(stream):
        if name == "gradient_fdfd256_nd4096":
            case = Wl.get_case("fdfd256")
            ctx = P.DbsContext(case, precision=P.PNGF_MIXED, device=str(dev), stream=stream)
            ctx.factor(Wl.random_design(case.n_d, 0))
            ctxs.append(ctx)
            g = torch.empty(case.n_d, dtype=torch.float64, device=dev)
            reps = 200

            def step():
                for _ in range(reps):
                    P.pngf_gradient(ctx.ctx, g.data_ptr(), None)
            units, unit, per = case.n_d * reps, "pixel gradients/s", reps
        else:
            base = "fdfd128_metal"
            tau = 1e-6 if name.startswith("pec") else args.tau
            if name.startswith("multifreq3"):
                cases = [Wl.get_case(base + "_l19"), Wl.get_case(base), Wl.get_case(base + "_l21")]
            else:
                cases = [Wl.get_case(base)]
            prec = P.PNGF_PEC if name.startswith("pec") else P.PNGF_FP64
            n = cases[0].n_d
            # independent searches (seeds 0 .. runs - 1) side by side, each a cooperative
            # launch of nsm / runs CTAs on its own stream
            n_side = max(1, args.side_runs)
            nsm = torch.cuda.get_device_properties(dev).multi_processor_count
            ctas = nsm // n_side if n_side > 1 else 0
            tiles = None
            if not name.startswith("pec"):
                tiles = (Wl.square_tiles(32, 32, 2) if name.startswith("tiles")
                         else np.arange(n, dtype=np.int32)[:, None])
            sets = []
            for i in range(n_side):
                s_i = torch.cuda.Stream(dev)
                b0 = Wl.random_design(n, i)
                cx_i = []
                for c in cases:
                    cx = P.DbsContext(c, precision=prec, tau=tau, refresh_k=args.refresh_k, device=str(dev),
                                      stream=s_i, n_ctas=ctas)
                    cx.factor(b0)
                    cx.snapshot()
                    cx_i.append(cx)
                    ctxs.append(cx)
                ts = P.TileSearch(cx_i, tiles, combine=P.PNGF_COMBINE_MEAN) if tiles is not None else None
                sets.append((s_i, cx_i, ts, torch.zeros(8, dtype=torch.int64, device=dev)))
            torch.cuda.synchronize(dev)
            if tiles is not None:
                ts0 = sets[0][2]
                extra["tile_m"], extra["n_tiles"], extra["systems"] = int(ts0.tile_m), int(ts0.n_tiles), len(cases)
            extra["runs"], extra["ctas_per_run"] = n_side, ctas if ctas else nsm

            def step():
                fork = torch.cuda.Event()
                fork.record(stream)
                for s_i, cx_i, ts, cnt_i in sets:
                    s_i.wait_event(fork)
                    for cx in cx_i:
                        P.pngf_restore(cx.ctx)
                    if ts is None:
                        P.pngf_dbs_sweep(cx_i[0].ctx, sweeps, None, None, None, 0, cnt_i.data_ptr())
                    else:
                        P.pngf_dbs_sweep_tiles([cx.ctx for cx in cx_i], ts.combine, ts.tiles.data_ptr(), ts.n_tiles,
                                               ts.tile_m, sweeps, None, None, None, 0, cnt_i.data_ptr(),
                                               ts.ws.data_ptr(), ts.ws_bytes)
                    j = torch.cuda.Event()
                    j.record(s_i)
                    stream.wait_event(j)
            unit, per = UNIT, n_side
        for _ in range(max(args.warmup, 1)):
            step()
        stream.synchronize()
        for cx in ctxs:
            if cx.sync() != 0:
                raise RuntimeError(f"{name}: warm-up failed")
        if name != "gradient_fdfd256_nd4096":
            c0 = sum(st[3].cpu().numpy() for st in sets)
            units = float(c0[1])
        torch.cuda.synchronize(dev)
        clocks = Clocks(dist.local)
        clocks.start()
        time.sleep(0.3)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            step()
        t1.record(stream)
        stream.synchronize()
        clk = clocks.stop()
    for cx in ctxs:
        if cx.sync() != 0:
            raise RuntimeError(f"{name}: timed steps failed")
    ms = t0.elapsed_time(t1) / args.steps
    value = units / (ms / 1e3)
    if name == "gradient_fdfd256_nd4096":
        n, n_o = 4096, 2
        bytes_per = n * ((n_o + 2) * 16 + 8)  # T rows, e, dv read; grad written
        gbs = bytes_per * reps / (ms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                "traffic": None, "kernel": "gradient_kernel",
                "note": "one launch reads (n_o + 2) x 16 B per pixel and writes 8 B (295 KB at N_d = 4096): "
                        "L2-resident and launch-latency bound, not a bandwidth test"}
        accepts = None
        extra["us_per_gradient"] = ms * 1e3 / reps
    else:
        c1 = sum(st[3].cpu().numpy() for st in sets)
        assert int(c1[1]) == int(c0[1]), "steps are not identical searches"
        accepts = int(c1[0])
        tri = n * (n + 1) / 2
        if name.startswith("pec"):
            flops = accepts * (2 * 8.0 * tri + 8.0 * n * n)  # W and H triangles, Q full: one complex FMA each
            kern = "dbs_pec_kernel"
        else:
            m = extra["tile_m"]
            flops = accepts * len(cases) * 8.0 * m * tri  # rank-m update of every system's triangle
            kern = "dbs_tiles_kernel"
        gf = flops / (ms / 1e3) / 1e9
        roof = {"bound": "alu", "achieved": gf / 1e3, "peak": peak_fp64 / 1e3, "unit": "TFLOP/s",
                "frac": gf / peak_fp64, "traffic": None, "kernel": kern,
                "peak_source": "FP64 FMA pipe, measured in this run by libpngf_peaks",
                "work": "complex FMAs of the kept flips' updates (8 real flop each)"}
    line = dict(metric=METRIC if unit == UNIT else "gradient throughput", value=value, unit=unit,
                n_gpus=dist.world, steps=args.steps, warmup=args.warmup, ms_per_step=ms, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                config={"workload": name, "what": SIDE_WORKLOADS[name], "max_sweeps": sweeps,
                        "step": ("restore the factored start + one search on each of %d concurrent runs" % per
                                 if unit == UNIT else "%d gradients" % per), **extra},
                roofline=roof, accepts_per_step=accepts, clocks=clk, gpu_launches=args.steps * per,
                cpu_baseline=None, e2e=None)
    if dist.rank == 0:
        print(json.dumps(line))
    for cx in ctxs:
        cx.close()
    return 0


# ---------------------------------------------------------------- GPU arm
class RunSet:
    """B independent DBS runs (seeds) on one device, each with its own context
    and persistent grid of ctas CTAs, dealt round-robin onto `slots` streams
    (default: one stream per run); a step forks from the timing stream, runs
    restore + pngf_dbs_sweep of every run on its slot's stream (the slots'
    cooperative launches execute side by side, a slot's runs one after another)
    and joins back."""

    def __init__(self, torch, P, Wl, case, dev, precision, args, seeds, ctas, tstream, inputs=None, slots=None):
        self.torch, self.P, self.case, self.dev, self.tstream = torch, P, case, dev, tstream
        self.n = case.n_d
        self.sweeps = args.sweeps
        self.trace_cap = args.sweeps * self.n
        self.slots = len(seeds) if slots is None else max(1, min(slots, len(seeds)))
        self.slot_streams = [torch.cuda.Stream(dev) for _ in range(self.slots)]
        self.streams = [self.slot_streams[i % self.slots] for i in range(len(seeds))]  # per run
        self.ctxs, self.traces, self.trace_f, self.counters = [], [], [], []
        self.factor_ms = []
        for i, seed in enumerate(seeds):
            s = self.streams[i]
            with torch.cuda.stream(s):
                kw = dict(precision=precision, tau=args.tau, refresh_k=args.refresh_k, device=str(dev), stream=s,
                          n_ctas=ctas)
                if precision == P.PNGF_MIXED:
                    kw.update(delay_r=args.delay_r, tensor_fold=args.tensor_fold)
                if inputs is not None:
                    kw["inputs_on_device"] = inputs
                c = P.DbsContext(case, **kw)
                if inputs is None:
                    inputs = (c.G, c.God, c.cd, c.co, c.dv)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                c.factor(Wl.random_design(self.n, seed=seed))
                e1.record(s)
                s.synchronize()
                self.factor_ms.append(e0.elapsed_time(e1))
                if c.sync() != 0:
                    raise P.PngfError(c.sync(), "pngf_factor")
                c.snapshot()
                self.ctxs.append(c)
                self.traces.append(torch.zeros((self.trace_cap, 4), dtype=torch.int32, device=dev))
                self.trace_f.append(torch.zeros(self.trace_cap, dtype=torch.float64, device=dev))
                self.counters.append(torch.zeros(8, dtype=torch.int64, device=dev))
        self.inputs = inputs
        self.kev = None

    def step(self, i_step=None, orders=None, subset=None):
        torch, P = self.torch, self.P
        fork = torch.cuda.Event()
        fork.record(self.tstream)
        for s in self.slot_streams:
            s.wait_event(fork)
        for r, (c, s) in enumerate(zip(self.ctxs, self.streams)):
            if subset is not None and r not in subset:
                continue
            P.pngf_restore(c.ctx)
            if i_step is not None:
                self.kev[i_step][r][0].record(s)
            P.pngf_dbs_sweep(c.ctx, self.sweeps, None if orders is None else orders[r], self.traces[r].data_ptr(),
                             self.trace_f[r].data_ptr(), self.trace_cap, self.counters[r].data_ptr())
            if i_step is not None:
                self.kev[i_step][r][1].record(s)
        for s in self.slot_streams:
            j = torch.cuda.Event()
            j.record(s)
            self.tstream.wait_event(j)

    def arm_events(self, steps):
        ev = self.torch.cuda.Event
        self.kev = [[(ev(enable_timing=True), ev(enable_timing=True)) for _ in self.ctxs] for _ in range(steps)]

    def counts(self):
        return np.stack([c.cpu().numpy() for c in self.counters])

    def status(self):
        return [c.sync() for c in self.ctxs]

    def close(self):
        for c in self.ctxs:
            c.close()


def autotune_launch(args, torch, P, Wl, case, dev, nsm, tstream):
    """Choose runs per GPU, the delay R and the fold engine of the mixed search
    from timed trials (paper_2501_18054_gb300.autotune): every trial's final
    designs must equal the FP64 path's from the same starts, with S within 1e-4."""
    import argparse
    from paper_2501_18054_gb300 import autotune as A
    cands = A.candidates(case.n_d, nsm, args.refresh_k, runs_options=(1, 2, 4, 6, 8), delay_options=(32, 64))
    max_runs = max(c.runs for c in cands)
    seeds = list(range(max_runs))
    ref = RunSet(torch, P, Wl, case, dev, P.PNGF_FP64, args, seeds, nsm // max_runs, tstream)
    ref.step()
    torch.cuda.synchronize(dev)
    if any(st != 0 for st in ref.status()):
        raise RuntimeError("autotune: FP64 reference runs failed")
    ref_out = [(cx.design(), (cx.eval_ports()[0] - case.s_off) * case.s_scale) for cx in ref.ctxs]
    inputs = ref.inputs
    ref.close()
    sets = {}
    for r in sorted({c.delay_r for c in cands}):
        a2 = argparse.Namespace(**vars(args))
        a2.delay_r = r
        sets[r] = RunSet(torch, P, Wl, case, dev, P.PNGF_MIXED, a2, seeds, nsm // max_runs, tstream, inputs=inputs)

    def measure(cand, steps):
        rs = sets[cand.delay_r]
        sub = set(range(cand.runs))
        for i in sub:
            rs.ctxs[i].set_launch(cand.ctas, cand.tensor_fold)
        rs.step(subset=sub)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(tstream)
        for _ in range(steps):
            rs.step(subset=sub)
        t1.record(tstream)
        torch.cuda.synchronize(dev)
        ok = all(rs.ctxs[i].sync() == 0 for i in sub)
        cnt = rs.counts()
        evals = float(sum(cnt[i, 1] for i in sub)) * steps
        same, err = True, 0.0
        for i in sub:
            b = rs.ctxs[i].design()
            same = same and bool(np.array_equal(b, ref_out[i][0]))
            if same:
                S = (rs.ctxs[i].eval_ports()[0] - case.s_off) * case.s_scale
                S_ref = ref_out[i][1]
                err = max(err, float(np.max(np.abs(S - S_ref) / np.maximum(np.abs(S_ref), 1e-3))))
        return A.Trial(cand, steps, evals / (t0.elapsed_time(t1) / 1e3), err, same, ok)

    win, trials = A.tune(cands, measure)
    for rs in sets.values():
        rs.close()
    return win, trials


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
    if args.workload == "hankel128_nd16384":
        return bench_hankel(args, torch, dist, dev, P, Wl)
    if args.workload in SIDE_WORKLOADS:
        return bench_side(args, torch, dist, dev, P, Wl)
    case = Wl.get_case(case_name(args.workload))
    n, n_o = case.n_d, case.n_o
    prec = P.PNGF_MIXED if args.precision == "mixed" else P.PNGF_FP64
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    tstream = torch.cuda.Stream(dev)
    tuned = None
    if prec == P.PNGF_MIXED and args.autotune:
        win, trials = autotune_launch(args, torch, P, Wl, case, dev, nsm, tstream)
        args.runs, args.delay_r, args.tensor_fold = win.cand.runs, win.cand.delay_r, win.cand.tensor_fold
        tuned = {"chosen": win.cand.as_dict(), "chosen_evals_per_s": win.evals_per_s, "bar": 1e-4,
                 "trials": [t.as_dict() for t in trials],
                 "note": "successive halving over runs per GPU x delay R x fold engine; every trial's final "
                         "designs equal the FP64 path's and S within 1e-4"}
    n_slots = max(1, args.runs)  # concurrent runs
    per_slot = max(1, args.runs_per_slot)
    n_runs = n_slots * per_slot  # runs per step
    ctas = args.ctas_per_run if args.ctas_per_run > 0 else (0 if n_slots == 1 else nsm // n_slots)
    seeds = replica_seeds(dist.rank, n_runs)
    rs = RunSet(torch, P, Wl, case, dev, prec, args, seeds, ctas, tstream, slots=n_slots)
    for _ in range(max(args.warmup, 1)):
        rs.step()
    torch.cuda.synchronize(dev)
    st = rs.status()
    if any(s != 0 for s in st):
        raise P.PngfError(max(st), "warm-up")
    c = rs.counts()
    evals_per_step, acc_per_step, sweeps_per_step = int(c[:, 1].sum()), int(c[:, 0].sum()), int(c[:, 2].sum())
    peak_fp64 = fp64_peak_gflops(tstream.cuda_stream)
    # ---- timed region (device time, CUDA events on the timing stream that forks and joins every run)
    rs.arm_events(args.steps)
    dist.barrier()
    torch.cuda.synchronize(dev)
    clocks = Clocks(dist.local)
    clocks.start()
    time.sleep(0.3)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(tstream)
    for i in range(args.steps):
        rs.step(i)
    t1.record(tstream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    dist.barrier()
    st = rs.status()
    if any(s != 0 for s in st):
        raise P.PngfError(max(st), "timed steps")
    c2 = rs.counts()
    assert int(c2[:, 1].sum()) == evals_per_step, "steps are not identical runs"
    cyc = rs.ctxs[0].phase_cycles()
    mhz = clk.get("sm_mhz") or 2070.0
    phase_names = ["score", "wait_after_score", "select_pivot_gather", "wait_or_flush",
                   "update", "refresh", "sweep_setup", "kernel_total", "refresh_x", "refresh_residual",
                   "refresh_correct", "refresh_ports", "publish", "update_delayed_sum",
                   "fold_prepare", "unused15"]
    phase_ms = {nm: float(cv) / (mhz * 1e3) for nm, cv in zip(phase_names, cyc)}
    ms = t0.elapsed_time(t1)
    ms_max = dist.max(torch, ms, dev)
    total_evals = dist.sum(torch, float(evals_per_step * args.steps), dev)
    value = total_evals / (ms_max / 1e3)
    kms = [a.elapsed_time(b) for per_step in rs.kev for a, b in per_step]
    k_avg = sum(kms) / len(kms)
    step_ms = ms / args.steps
    peaks = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    tri = n * (n + 1) / 2
    runs_note = ("%d runs per step, %d at a time (%d streams of %d cooperative launches one after another, "
                 "%d CTAs each): achieved = the launches' algorithmic work per step / device time of a step"
                 % (n_runs, n_slots, n_slots, per_slot, ctas or nsm)) if n_runs > 1 else None
    if prec == P.PNGF_FP64:
        # dominant kernel: the persistent FP64 DBS sweep.  Algorithmic work per
        # launch: the rank-1 update of the upper triangle of W per kept flip,
        # 4 DFMA = 8 flop per complex element (32 bytes of W read + written).
        flops = acc_per_step * 8.0 * tri
        bytes_w = acc_per_step * 32.0 * tri
        achieved_gflops = flops / (step_ms / 1e3) / 1e9
        roofline = {"bound": "alu", "achieved": achieved_gflops / 1e3, "peak": peak_fp64 / 1e3,
                    "unit": "TFLOP/s", "frac": achieved_gflops / peak_fp64, "traffic": None,
                    "kernel": "dbs_fp64_kernel",
                    "peak_source": "FP64 FMA pipe, measured in this run by libpngf_peaks "
                                   "(152 SMs x 2 DFMA/clk x 2 flop x clock)",
                    "hbm_view": {"achieved_gbs": bytes_w / (step_ms / 1e3) / 1e9, "peak_gbs": hbm_peak,
                                 "frac": bytes_w / (step_ms / 1e3) / 1e9 / hbm_peak,
                                 "peak_source": "MEASURED_PEAKS.json hbm_gbs"}}
    else:
        # dominant kernel: the persistent mixed DBS sweep.  Algorithmic HBM bytes per
        # launch: per flush the upper triangle of the two FP32 planes read + written
        # (16 B per element); per refresh with m active pixels the m rows of G as FP32
        # pairs (16 B x m x n), the FP32 upper triangle (8 B) and its entries in the
        # active rows above each column strip (8 B x m / n per element); per kept flip
        # one column of the FP32 planes (8 B x n); per evaluation (3 + n_o) x 16 B of
        # FP64 state.
        bytes_alg = mixed_alg_bytes(c2, n, n_o)
        gbs = bytes_alg / (step_ms / 1e3) / 1e9
        traffic, traffic_note = None, "no capture of the current kernel sources"
        if args.workload == TRAFFIC_CAPTURE["workload"] and sources_fingerprint() == TRAFFIC_CAPTURE["sources_sha256"]:
            ratio = TRAFFIC_CAPTURE["measured_bytes"] / TRAFFIC_CAPTURE["algorithmic_bytes"]
            traffic = ratio * bytes_alg
            traffic_note = ("bytes per step: ncu dram read + write of one captured launch (one run, seed 0, "
                            "19 CTAs: the headline launch shape) = %.3f x its algorithmic bytes, scaled to "
                            "this step's algorithmic bytes" % ratio)
        roofline = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                    "traffic": traffic, "traffic_note": traffic_note, "algorithmic_bytes_per_step": bytes_alg,
                    "kernel": "dbs_mixed_kernel",
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst copy)",
                    "note": "each run keeps one flip at a time (a latency-bound chain of word exchange, "
                            "fetch and FP64 state update per kept flip) and refreshes e, T with a double-float "
                            "residual (FP32-pipe bound); see phase_ms_cta0"}
    if runs_note:
        roofline["runs"] = runs_note
    # ---- end to end through the C ABI with host buffers (pinned): visiting orders in,
    #      traces, objective values, counters and port amplitudes out, every step
    e2e = None
    if not args.no_e2e:
        order_h = torch.from_numpy(np.tile(np.arange(n, dtype=np.int32), (args.sweeps, 1))).pin_memory()
        orders_d = [torch.empty_like(order_h, device=dev) for _ in rs.ctxs]
        outs = [(torch.empty((rs.trace_cap, 4), dtype=torch.int32).pin_memory(),
                 torch.empty(rs.trace_cap, dtype=torch.float64).pin_memory(),
                 torch.empty(8, dtype=torch.int64).pin_memory()) for _ in rs.ctxs]
        h2d = order_h.numel() * 4 * n_runs
        d2h = (outs[0][0].numel() * 4 + outs[0][1].numel() * 8 + 64 + 16 * n_o + 8) * n_runs
        for rep in range(2):
            dist.barrier()
            torch.cuda.synchronize(dev)
            w0 = time.perf_counter()
            for i in range(args.steps):
                for r, s in enumerate(rs.streams):
                    with torch.cuda.stream(s):
                        orders_d[r].copy_(order_h, non_blocking=True)
                for r, s in enumerate(rs.streams):  # the step forks after every run's copy
                    ev = torch.cuda.Event()
                    ev.record(s)
                    tstream.wait_event(ev)
                rs.step(None, [o.data_ptr() for o in orders_d])
                for r, s in enumerate(rs.streams):
                    with torch.cuda.stream(s):
                        outs[r][0].copy_(rs.traces[r], non_blocking=True)
                        outs[r][1].copy_(rs.trace_f[r], non_blocking=True)
                        outs[r][2].copy_(rs.counters[r], non_blocking=True)
                for cx in rs.ctxs:
                    cx.eval_ports()  # synchronizes: each run's result on the host
            w1 = time.perf_counter()
        assert sum(int(o[2][1]) for o in outs) == evals_per_step
        e2e_s = dist.max(torch, w1 - w0, dev)
        e2e = {"value": total_evals / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}
    # ---- the same runs on the FP64 path (same GPU, same starts, same concurrency)
    #      for the speedup and the S-parameter error of the mixed path
    rs.step()
    torch.cuda.synchronize(dev)
    res_main = [(cx.eval_ports()[0], cx.design(), rs.traces[r][:min(int(c2[r, 0]), rs.trace_cap), 2].cpu().numpy())
                for r, cx in enumerate(rs.ctxs)]
    compare = None
    if prec == P.PNGF_MIXED and not args.no_fp64_compare:
        ref = RunSet(torch, P, Wl, case, dev, P.PNGF_FP64, args, seeds, ctas, tstream, inputs=rs.inputs,
                     slots=n_slots)
        ref.step()
        torch.cuda.synchronize(dev)
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 2
        r0.record(tstream)
        for _ in range(reps):
            ref.step()
        r1.record(tstream)
        torch.cuda.synchronize(dev)
        if any(s != 0 for s in ref.status()):
            raise RuntimeError("FP64 comparison runs failed")
        c64 = ref.counts()
        ms64 = r0.elapsed_time(r1) / reps
        ev64 = float(c64[:, 1].sum()) / (ms64 / 1e3)
        same_all, prefix_min, s_err = True, None, 0.0
        for r, cx in enumerate(ref.ctxs):
            o64 = cx.eval_ports()[0]
            b64 = cx.design()
            k64 = ref.traces[r][:min(int(c64[r, 0]), ref.trace_cap), 2].cpu().numpy()
            o_m, b_m, k_m = res_main[r]
            same = bool(np.array_equal(b64, b_m))
            same_all = same_all and same
            prefix = next((i for i, (x, y) in enumerate(zip(k64, k_m)) if x != y), min(len(k64), len(k_m)))
            prefix_min = prefix if prefix_min is None else min(prefix_min, prefix)
            if same:
                S_m = (o_m - case.s_off) * case.s_scale
                S_64 = (o64 - case.s_off) * case.s_scale
                s_err = max(s_err, float(np.max(np.abs(S_m - S_64) / np.maximum(np.abs(S_64), 1e-3))))
        compare = {"fp64_evals_per_s": ev64, "fp64_ms_per_step": ms64, "speedup_vs_fp64": value / ev64,
                   "same_final_design": same_all, "identical_accept_prefix_min": int(prefix_min),
                   "accepts_fp64": int(c64[:, 0].sum()), "accepts_mixed": int(acc_per_step),
                   "runs_compared": n_runs}
        if same_all:
            compare["s_param_max_rel_err_vs_fp64"] = s_err
        ref.close()
    if dist.rank == 0:
        import oracle as O
        p = O.Problem.from_case(case)
        err = 0.0
        for o_m, b_m, _ in res_main:
            ev = O.evaluate(p, b_m)
            S_exact = (ev.o - case.s_off) * case.s_scale
            S_m = (o_m - case.s_off) * case.s_scale
            err = max(err, float(np.max(np.abs(S_m - S_exact) / np.maximum(np.abs(S_exact), 1e-3))))
        compare = dict(compare or {})
        compare["s_param_max_rel_err_vs_oracle"] = err
        compare["s_param_err_note"] = ("final design of every timed run, exact S from the CPU FP64 oracle "
                                       "(relative to max(|S|, 1e-3))")
    cpu = None
    if dist.rank == 0 and not args.no_cpu_baseline:
        v, m, dt = time_oracle(case, Wl.random_design(n, seed=seeds[0]), args.cpu_sample_evals)
        cpu = {"value": v, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
               "sample": f"first {m} attempted flips of the same raster DBS run, each re-solved with "
                         f"LAPACK zgesv at n={n} ({dt:.1f} s)"}
        if args.cpu_one_core:
            cpu["one_core"] = time_oracle_one_core(args.workload, 1)
        pv, pe, pk, pdt, pfac = time_paper_algorithm(case, Wl.random_design(n, seed=seeds[0]), args.cpu_kept_flips)
        cpu["paper_algorithm"] = {"value": pv, "unit": UNIT, "cores": blas_threads(),
                                  "kind": "the paper's Sherman-Morrison DBS in numpy + threaded BLAS",
                                  "sample": f"first {pk} kept flips ({pe} attempted) of the same run, "
                                            f"{pdt:.1f} s; its factor {pfac:.1f} s (not counted)"}
    if dist.rank == 0:
        line = dict(
            metric=METRIC, value=value, unit=UNIT, n_gpus=dist.world, steps=args.steps, warmup=args.warmup,
            ms_per_step=ms_max / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
            dtype="f64" if prec == P.PNGF_FP64 else "f32+f64", data="synthetic",
            config={"workload": args.workload, "n_d": n, "n_o": n_o, "precision": args.precision,
                    "runs_per_gpu": n_runs, "concurrent_runs": n_slots, "runs_per_slot": per_slot,
                    "ctas_per_run": ctas if ctas else nsm,
                    "seeds": seeds,
                    "mode": "first-improvement, raster order", "max_sweeps": args.sweeps,
                    "refresh_k": args.refresh_k, "tau": args.tau,
                    "delay_r": args.delay_r if prec == P.PNGF_MIXED else None,
                    "fold": ("tcgen05 3xTF32" if args.tensor_fold else "FP32 CUDA cores")
                    if prec == P.PNGF_MIXED else None,
                    "step": "restore every run's factored start state + DBS for up to %d sweeps or until "
                            "a sweep keeps no flip; %d runs at a time, %d after one another on each of %d "
                            "streams" % (args.sweeps, n_slots, per_slot, n_slots),
                    "l2": "inputs larger than L2 (W = %.0f MB complex128 per run)" % (n * n * 16 / 1e6),
                    "replicas": "independent runs per GPU (seed = rank * runs + i)"},
            roofline=roofline, cpu_baseline=cpu, e2e=e2e, clocks=clk, gpu_launches=args.steps * n_runs,
            evals_per_step=evals_per_step, accepts_per_step=acc_per_step, sweeps_per_step=sweeps_per_step,
            accepts_per_s=acc_per_step * args.steps / (ms_max / 1e3),
            sweeps_per_s=sweeps_per_step * args.steps / (ms_max / 1e3),
            kernel_ms_avg=k_avg, factor_ms=statistics.mean(rs.factor_ms), fp64_peak_gflops=peak_fp64,
            phase_ms_cta0=phase_ms, mixed_vs_fp64=compare, autotune=tuned)
        print(json.dumps(line))
    rs.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
