"""The GPU path's fixed-point numerator accumulators (fixed192.cuh: 192- and
128-bit), compiled for the host, against exact rational arithmetic (CPU)."""
import os
import random
import struct
import subprocess
from fractions import Fraction

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    exe = tmp_path_factory.mktemp("fx") / "fx192"
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-o", str(exe),
                           os.path.join(HERE, "fixed192_harness.cpp")])
    return str(exe)


def _bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def _dbl(b):
    return struct.unpack("<d", struct.pack("<Q", b))[0]


def _exact_rounded(vals, lead=166):
    """Round each value to the run's grid, sum exactly, round to double.

    The grid is 2^(e - lead) where 2^e <= max|x| < 2^(e+1) (e of the run's largest
    normal exponent; subnormals and zeros count as 2^-1022); lead is 166 for the
    192-bit accumulator and 100 for the 128-bit one.
    """
    import math
    e = -1022
    for v in vals:
        if v != 0.0:
            e = max(e, math.frexp(abs(v))[1] - 1)
    q = Fraction(2) ** (e - lead)
    tot = Fraction(0)
    for v in vals:
        f = Fraction(v) / q
        n = round(f)  # Python rounds half to even
        tot += n * q
    return float(tot)  # correctly rounded (ties to even)


def _run(exe, groups, width=192):
    inp = "".join(f"{len(g)} " + " ".join(f"{_bits(x):x}" for x in g) + "\n" for g in groups)
    args = [exe] + (["128"] if width == 128 else [])
    out = subprocess.run(args, input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    res = []
    for line in out:
        if line.strip():
            h, o = line.split()
            res.append((_dbl(int(h, 16)), int(o)))
    return res


@pytest.mark.parametrize("width,lead", [(192, 166), (128, 100)])
def test_exact_sum_matches_rationals(harness, width, lead):
    rng = random.Random(7)
    groups = []
    for _ in range(400):
        k = rng.choice([1, 2, 3, 7, 30, 200])
        scale = 10.0 ** rng.uniform(-30, 2)
        g = [rng.choice([-1, 1]) * rng.random() * scale * 10.0 ** rng.uniform(-8, 0) for _ in range(k)]
        groups.append(g)
    # cancellation, tiny tails, exact ties and signed zeros
    groups += [[1.0, -1.0], [1e-300, 1.0, -1.0], [2.0 ** 60, 1.0, -(2.0 ** 60)],
               [0.1, 0.2, -0.3], [-0.0], [0.0, -0.0], [3.0 * 2.0 ** -130], [2.0 ** -129],
               [1e-40, -1e-40, 1e-200], [1e-36, -0.9e-36, 3e-52],
               [1.0, 1.5 * 2.0 ** -167], [1.0, 2.5 * 2.0 ** -167], [1.0, 2.0 ** -200],
               [1e-310, 2e-310, -1e-311], [1e300, -1e300, 1e200]]
    res = _run(harness, groups, width)
    for g, (got, ovf) in zip(groups, res):
        assert ovf == 0
        want = _exact_rounded(g, lead)
        assert got == want or (got == 0.0 and want == 0.0), (g[:4], got, want)


@pytest.mark.parametrize("width", [192, 128])
def test_order_independent(harness, width):
    rng = random.Random(3)
    g = [rng.uniform(-1, 1) * 10.0 ** rng.uniform(-15, 1) for _ in range(1000)]
    perms = [g, list(reversed(g)), sorted(g), sorted(g, key=abs)]
    res = _run(harness, perms, width)
    assert len({r[0] for r in res}) == 1


@pytest.mark.parametrize("width", [192, 128])
def test_overflow_flagged(harness, width):
    res = _run(harness, [[float("inf")], [2.0 ** 1000, 2.0 ** 1000], [1e308, 1e308]], width)
    assert res[0][1] == 1 and res[1][1] == 0 and res[2][1] == 0
    assert res[1][0] == 2.0 ** 1001
