"""Write the stored expected DBS trajectories under tests/golden/.

Every value here comes from the CPU oracle (``oracle/``) run on the seeded
synthetic inputs of ``paper_2501_18054_gb300.workloads``; nothing is taken
from the CUDA path.  Re-run after a change to the oracle or the inputs:

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from paper_2501_18054_gb300 import workloads as W  # noqa: E402
import oracle as O  # noqa: E402

RUNS = {
    # 64^2 FDFD, 10x10 design in {1, 4}, random p=0.5 start (seed 0), 3 raster sweeps, maximise |T21|^2
    "fdfd64_first_raster": dict(case="fdfd64", seed=0, n_sweeps=3, order="raster", mode=O.FIRST_IMPROVEMENT),
    "fdfd64_first_shuffled": dict(case="fdfd64", seed=0, n_sweeps=6, order="shuffled", mode=O.FIRST_IMPROVEMENT),
    "fdfd64_best": dict(case="fdfd64", seed=1, n_sweeps=200, order="raster", mode=O.BEST_IMPROVEMENT),
}
TAU = 1e-9


def order_for(spec, n_d):
    if spec["order"] == "raster":
        return W.raster_order(n_d, spec["n_sweeps"])
    return W.shuffled_order(n_d, spec["n_sweeps"], seed=spec["seed"])


def main():
    for name, spec in RUNS.items():
        case = W.get_case(spec["case"])
        p = O.Problem.from_case(case)
        b0 = W.random_design(case.n_d, spec["seed"])
        res = O.dbs(p, b0, order_for(spec, case.n_d), tau=TAU, mode=spec["mode"])
        out = dict(
            run=name, spec=spec, tau=TAU, n_d=case.n_d,
            accepted=[[int(s), int(t), int(k), float(f)] for (s, t, k, f) in res.accepted],
            final_b=res.b.astype(int).tolist(), final_f=res.f,
            final_o=[[float(z.real), float(z.imag)] for z in res.o],
            n_evals=res.n_evals, sweeps_done=res.sweeps_done, min_abs_margin=res.min_abs_margin,
            source="oracle.dbs (re-solve of every candidate with LAPACK zgesv, FP64)",
        )
        with open(os.path.join(HERE, f"{name}.json"), "w") as fh:
            json.dump(out, fh, indent=1)
        print(name, len(res.accepted), "accepts", res.sweeps_done, "sweeps", "f", res.f)


if __name__ == "__main__":
    main()
