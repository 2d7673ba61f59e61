"""Autotuner of the mixed-precision search's launch configuration.

The method fixes what is computed; how the search is laid out on the GPU is
free and is chosen here from timed trials:

* ``runs``        independent searches (random starts) side by side on one GPU,
                  each a cooperative launch of ``n_sm // runs`` CTAs;
* ``delay_r``     kept flips between two folds of the delayed set into the FP32
                  inverse (a divisor of the refresh interval, so that a refresh
                  follows a fold);
* ``tensor_fold`` the fold on the tensor cores (tcgen05, 3xTF32) or on the FP32
                  CUDA cores.

A candidate is admissible when its launch can hold the region: the mixed
search keeps each CTA's share of the pixels in shared memory (at most
``own_max`` = 256 per CTA), and between folds their delayed rows and partial
sums, (R + 8) x own (rounded up to 32) x 8 bytes, in a 144 KB work area.  A
trial is accurate when every run ends on the same final design as the FP64
path from the same start and its S-parameters are within the accuracy bar
(1e-4 relative) of the FP64 path's; only accurate trials are eligible.  The search is successive halving: every
candidate is timed briefly, the fastest third is timed again with more steps,
and the fastest of those wins (ties: fewer runs, then the smaller delay, then
the tensor-core fold).

This module holds host logic only; the measurement is a callable the caller
supplies (``bench.py`` times real searches through the C ABI).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Iterable, List, Optional, Sequence


@dataclasses.dataclass(frozen=True)
class Candidate:
    runs: int
    ctas: int
    delay_r: int
    tensor_fold: int

    def as_dict(self) -> dict:
        return dataclasses.asdict(self)


@dataclasses.dataclass
class Trial:
    cand: Candidate
    steps: int
    evals_per_s: float
    s_err: float  # largest relative S-parameter error of the runs against the FP64 path
    same_design: bool  # every run ended on the FP64 path's final design
    ok: bool = True  # the launches returned PNGF_OK

    def accurate(self, bar: float) -> bool:
        return self.ok and self.same_design and self.s_err <= bar

    def as_dict(self) -> dict:
        d = self.cand.as_dict()
        d.update(steps=self.steps, evals_per_s=self.evals_per_s, s_err=self.s_err,
                 same_design=self.same_design, ok=self.ok)
        return d


WORK_BYTES = 147456  # the mixed search's shared-memory work area
PARTS_MAX = 8


def delayed_fits(n_d: int, ctas: int, r: int, work_bytes: int = WORK_BYTES) -> bool:
    """The delayed rows (r per pixel) and the delayed sum's partials of the
    largest CTA share fit in the work area."""
    own = -(-n_d // ctas)
    oss = (own + 31) // 32 * 32
    return (r + PARTS_MAX) * oss * 8 <= work_bytes


def candidates(n_d: int, n_sm: int, refresh_k: int, runs_options: Sequence[int] = (1, 2, 3, 4),
               delay_options: Sequence[int] = (32, 64), fold_options: Sequence[int] = (1, 0),
               own_max: int = 256, max_delay: int = 128) -> List[Candidate]:
    """Every admissible launch configuration, in a fixed order."""
    out = []
    for runs in runs_options:
        ctas = n_sm // runs
        if runs < 1 or ctas < 1 or n_d > own_max * ctas:
            continue
        for r in delay_options:
            if r < 1 or r > max_delay or (refresh_k > 0 and refresh_k % r) or not delayed_fits(n_d, ctas, r):
                continue
            for fold in fold_options:
                out.append(Candidate(runs, ctas, r, int(fold)))
    return out


def _key(t: Trial):
    # faster first; ties: fewer runs, smaller delay, tensor-core fold
    return (-t.evals_per_s, t.cand.runs, t.cand.delay_r, -t.cand.tensor_fold)


def select(trials: Iterable[Trial], bar: float = 1e-4) -> Trial:
    """The fastest accurate trial; ValueError when none is accurate."""
    good = [t for t in trials if t.accurate(bar)]
    if not good:
        raise ValueError("no trial meets the accuracy bar")
    return sorted(good, key=_key)[0]


def tune(cands: Sequence[Candidate], measure: Callable[[Candidate, int], Trial], bar: float = 1e-4,
         first_steps: int = 1, final_steps: int = 3, keep_frac: float = 1.0 / 3.0,
         log: Optional[list] = None):
    """Successive halving over ``cands``; returns (winner, every trial run).

    ``measure(cand, steps)`` times ``steps`` steps of the search in that
    configuration and reports its accuracy.
    """
    if not cands:
        raise ValueError("no admissible candidate")
    trials = [measure(c, first_steps) for c in cands]
    good = sorted([t for t in trials if t.accurate(bar)], key=_key)
    if not good:
        raise ValueError("no candidate meets the accuracy bar")
    keep = max(1, int(math.ceil(len(good) * keep_frac)))
    finals = [measure(t.cand, final_steps) for t in good[:keep]]
    everything = trials + finals
    if log is not None:
        log.extend(t.as_dict() for t in everything)
    return select(finals, bar), everything
