"""The double-float building blocks of the CUDA library, checked on the CPU.

``paper_2008_03276_gb300/csrc/df64.cuh`` is compiled for the host by
``tests/host/df64_host.cpp`` with the CUDA float intrinsics replaced by the host's IEEE
binary32 operations (same rounding: nearest-even, fused multiply-add rounded once).  Every
result is compared with exact rational arithmetic (``fractions.Fraction``).  Inputs come from
the float64 -> double-float split, whose ``hi`` is the truncated leading 24 bits, so
``|lo| < ulp(hi) <= 2u |hi|`` (u = 2^-24) rather than the ``u |hi|`` of a rounded split; the
bounds below are derived for such inputs by summing the roundings of each step:

* ``df_mul_f`` (df x float): one rounded FMA after an exact product, <= 3u^2 relative;
* ``df_add`` (sloppy addition): <= 9u^2 (|x| + |y|) absolute, cancellation included;
* ``df_mul``: two rounded FMAs and the neglected lo*lo term, <= 12u^2 relative;
* ``df_div``, ``df_rcp`` (float quotient plus one correction): <= 24u^2 relative;
* ``df_sub_two_prods`` (z - ab - cd, one renormalisation): <= 32u^2 (|z| + |ab| + |cd|).

A dropped term or a wrong sign in any of them shows as an error of order u, far above these.
The split itself: ``hi`` is the exact truncation, ``lo`` the nearest float to the remainder in
the branch-free window 2^-74 <= |d| < 2^128, within 2^-47 |d| elsewhere down to 2^-100, below
which values flush to zero; infinities and NaN keep their kind.
"""
import math
import os
import shutil
import struct
import subprocess
from fractions import Fraction as F

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
U2 = F(1, 2**48)


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("df64") / "df64_host")
    subprocess.run([cxx, "-O2", "-ffp-contract=off", "-std=c++17", "-I", os.path.join(ROOT, "tests", "host", "stub"),
                    "-I", os.path.join(ROOT, "paper_2008_03276_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host", "df64_host.cpp"), "-o", exe], check=True)
    return exe


def run(exe, op, n, seed):
    out = subprocess.run([exe, op, str(n), str(seed)], capture_output=True, text=True, check=True).stdout
    return [line.split() for line in out.splitlines()]


def f32(h):
    return struct.unpack("<f", struct.pack("<I", int(h, 16)))[0]


def f64(h):
    return struct.unpack("<d", struct.pack("<Q", int(h, 16)))[0]


def dfv(hi, lo):
    return F(f32(hi)) + F(f32(lo))


def nearest_float(q):
    """The binary32 value nearest to the rational q (ties to even), for |q| in the normal range."""
    if q == 0:
        return 0.0
    s = -1 if q < 0 else 1
    q = abs(q)
    e = math.floor(math.log2(q))
    while F(2) ** e > q:
        e -= 1
    while F(2) ** (e + 1) <= q:
        e += 1
    scale = F(2) ** (e - 23)
    m = q / scale  # in [2^23, 2^24)
    r = math.floor(m)
    frac = m - r
    if frac > F(1, 2) or (frac == F(1, 2) and r % 2 == 1):
        r += 1
    return s * float(r * scale)


def truncate24(d):
    """d with its significand cut to the leading 24 bits (toward zero)."""
    m, e = math.frexp(abs(d))  # m in [0.5, 1)
    t = math.floor(m * 2**24) / 2**24
    return math.copysign(math.ldexp(t, e), d)


def test_split_of_float64(harness):
    rows = run(harness, "from_double", 40000, 11)
    for dh, hh, lh in rows:
        d, hi, lo = f64(dh), f32(hh), f32(lh)
        if math.isnan(d):
            assert math.isnan(hi) and lo == 0.0
            continue
        if math.isinf(d):
            assert hi == d and lo == 0.0
            continue
        a = abs(d)
        if a < 2.0**-100:
            assert hi == 0.0 and lo == 0.0 and math.copysign(1.0, hi) == math.copysign(1.0, d)
            continue
        if a >= 2.0**128:
            assert math.isinf(hi) and math.copysign(1.0, hi) == math.copysign(1.0, d) and lo == 0.0
            continue
        assert hi == truncate24(d), dh
        assert lo == 0.0 or math.copysign(1.0, lo) == math.copysign(1.0, d)
        err = abs(F(hi) + F(lo) - F(d))
        assert err <= F(1, 2**47) * F(a), dh
        if 2.0**-74 <= a:
            assert lo == nearest_float(F(d) - F(hi)), dh


def test_branch_free_split_is_the_same_split(harness):
    """df_from_double_sel (no branches, for long straight-line kernels) returns the bits of
    df_from_double on every input class the split test draws (fast window, all of float64, the
    flush edge, zeros, infinities, NaN, the range limits)."""
    a = run(harness, "from_double", 40000, 11)
    b = run(harness, "from_double_sel", 40000, 11)
    assert a == b


@pytest.mark.parametrize("op,bound", [("add", 9), ("mul", 12), ("div", 24), ("mul_f", 3)])
def test_binary_operations_within_their_bounds(harness, op, bound):
    worst = F(0)
    for t in run(harness, op, 20000, 5):
        if op == "mul_f":
            x, y, r = dfv(t[0], t[1]), F(f32(t[2])), dfv(t[3], t[4])
        else:
            x, y, r = dfv(t[0], t[1]), dfv(t[2], t[3]), dfv(t[4], t[5])
        if op == "add":
            e = abs(r - (x + y)) / (abs(x) + abs(y))
        elif op in ("mul", "mul_f"):
            e = abs(r - x * y) / abs(x * y)
        else:
            e = abs(r - x / y) / abs(x / y)
        worst = max(worst, e)
        # the result is a renormalised pair: |lo| <= ulp(hi) / 2
        rh, rl = f32(t[-2]), f32(t[-1])
        assert abs(rl) <= abs(rh) * 2.0**-24
    assert worst <= bound * U2, float(worst / U2)


def test_reciprocal_within_its_bound(harness):
    worst = F(0)
    for t in run(harness, "rcp", 20000, 6):
        y, r = dfv(t[0], t[1]), dfv(t[2], t[3])
        worst = max(worst, abs(r * y - 1))
    assert worst <= 24 * U2, float(worst / U2)


def test_two_products_subtracted_within_its_bound(harness):
    worst = F(0)
    for t in run(harness, "sub_two_prods", 20000, 7):
        z, a, b, c, d, r = [dfv(t[2 * i], t[2 * i + 1]) for i in range(6)]
        worst = max(worst, abs(r - (z - a * b - c * d)) / (abs(z) + abs(a * b) + abs(c * d)))
    assert worst <= 32 * U2, float(worst / U2)


def test_error_free_products_are_exact_on_floats(harness):
    """With lo = 0 on both sides, df_mul returns the exact product of two floats (TwoProd by
    FMA: the product of two 24-bit significands fits in the pair), as long as its low part does
    not underflow (factors between 2^-40 and 2^41 here)."""
    rows = run(harness, "mul_floats", 20000, 8)
    assert len(rows) == 20000
    for t in rows:
        assert dfv(t[4], t[5]) == F(f32(t[0])) * F(f32(t[2]))
