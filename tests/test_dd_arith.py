"""Double-float arithmetic of the mixed search (csrc/dd.cuh), compiled for the
host and checked against exact rational arithmetic.

Bars (u = 2^-24): the accurate double-word sum within 3 u^2 of the exact sum,
also under cancellation; products within 5 u^2 (two double-words) and 2 u^2
(a double-word and a float); reciprocal and square root within 8 u^2 (one
Newton step from the correctly rounded FP32 value); every result normalised
(|lo| <= ulp(hi) / 2); the comparison exact on normalised pairs.
"""
import os
import shutil
import struct
import subprocess
from fractions import Fraction as F

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2501_18054_gb300", "csrc")
U2 = F(1, 2 ** 48)


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("dd") / "dd_host_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC,
                    os.path.join(HERE, "dd_host_check.cpp"), "-o", out], check=True)
    return out


def fbits(x):
    return struct.unpack("<I", struct.pack("<f", np.float32(x)))[0]


def bfloat(u):
    return struct.unpack("<f", struct.pack("<I", u))[0]


def val(p):
    return F(p[0]) + F(p[1])


def make_dd(rng, scale=1.0):
    """a normalised double-word from a random FP64 value"""
    x = rng.standard_normal() * scale * np.exp(rng.uniform(-3, 3))
    hi = np.float32(x)
    lo = np.float32(x - np.float64(hi))
    return (float(hi), float(lo))


def run(exe, lines):
    inp = "".join("%s %08x %08x %08x %08x\n" % (op, fbits(a[0]), fbits(a[1]), fbits(b[0]), fbits(b[1]))
                  for op, a, b in lines)
    res = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    out = []
    for ln in res:
        if ln.strip():
            h, l = ln.split()
            out.append((bfloat(int(h, 16)), bfloat(int(l, 16))))
    return out


def normalised(p):
    hi, lo = p
    if hi == 0.0:
        return lo == 0.0
    ulp = np.spacing(np.float32(abs(hi)))
    return abs(lo) <= ulp / 2


def check(exe, op, pairs, exact, bound):
    out = run(exe, [(op, a, b) for a, b in pairs])
    worst = F(0)
    for (a, b), z in zip(pairs, out):
        e = exact(a, b)
        assert normalised(z), (op, a, b, z)
        if e != 0:
            worst = max(worst, abs(val(z) - e) / abs(e))
    assert worst <= bound, (op, float(worst), float(bound))
    return float(worst)


def test_add_sub(exe):
    rng = np.random.default_rng(1)
    pairs = [(make_dd(rng), make_dd(rng)) for _ in range(400)]
    # cancellation: y close to -x
    for _ in range(200):
        x = make_dd(rng)
        d = make_dd(rng, 1e-5)
        v = -(np.float64(x[0]) + np.float64(x[1])) + (d[0] + d[1]) * abs(x[0])
        hi = np.float32(v)
        pairs.append((x, (float(hi), float(np.float32(v - np.float64(hi))))))
    check(exe, "add", pairs, lambda a, b: val(a) + val(b), 3 * U2)
    check(exe, "sub", pairs, lambda a, b: val(a) - val(b), 3 * U2)


def test_mul(exe):
    rng = np.random.default_rng(2)
    pairs = [(make_dd(rng), make_dd(rng)) for _ in range(400)]
    check(exe, "mul", pairs, lambda a, b: val(a) * val(b), 5 * U2)
    pf = [(a, (b[0], 0.0)) for a, b in pairs]
    check(exe, "mulf", pf, lambda a, b: val(a) * F(b[0]), 2 * U2)


def test_rcp_sqrt(exe):
    rng = np.random.default_rng(3)
    xs = [make_dd(rng) for _ in range(400)]
    check(exe, "rcp", [(x, (0.0, 0.0)) for x in xs], lambda a, b: 1 / val(a), 8 * U2)
    pos = [(abs(x[0]), abs(x[1]) if x[0] * x[1] >= 0 else -abs(x[1])) for x in xs]
    out = run(exe, [("sqrt", x, (0.0, 0.0)) for x in pos])
    for x, z in zip(pos, out):
        assert normalised(z)
        # (s_hi + s_lo)^2 against x, relative: 2 x the bound on s
        assert abs(val(z) ** 2 - val(x)) / val(x) <= 16 * U2, (x, z)


def test_compare(exe):
    rng = np.random.default_rng(4)
    pairs = []
    for _ in range(300):
        x = make_dd(rng)
        if rng.uniform() < 0.5:  # equal hi parts, different lo parts
            lo = float(np.float32(x[1] * rng.uniform(-1, 1)))
            pairs.append((x, (x[0], lo)))
        else:
            pairs.append((x, make_dd(rng)))
    out = run(exe, [("gt", a, b) for a, b in pairs])
    for (a, b), z in zip(pairs, out):
        assert (z[0] == 1.0) == (val(a) > val(b)), (a, b)
