"""The FP64 form's slice arithmetic (the integer digit split and the single
rounding of an exact level sum: paper_1301_0191_gb300/csrc/oz_arith.h, the
same code the tensor-core kernels run) built for the host and checked against
exact rational arithmetic:

  * digits: x = 2^e sum_p m_p 2^-7(p+1) within 2^-57 2^e, |m_0| <= 128,
    |m_p| <= 64, 2^(e-1) <= max |x| < 2^e (zeros, subnormals, huge and tiny
    rows, mixed signs);
  * exactness of the level sums: for K = 256 and digits at their bounds, every
    level's sum of slice products stays below 2^24 (so the FP32 tensor-core
    accumulation is exact);
  * rounding: (H 2^28 + L) 2^s rounded to the nearest double, ties to even,
    equals Python's correctly rounded conversion of the exact rational, for
    cancelling and non-cancelling (H, L), and at the edges of the normal
    range.
"""
import os
import random
import shutil
import struct
import subprocess
from fractions import Fraction

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1301_0191_gb300", "csrc")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("oz") / "harness")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "slice_arith_harness.cpp"), "-o", exe],
                   check=True)
    return exe


def _run(exe, text):
    return subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout.split("\n")


def _bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def _double(u):
    return struct.unpack("<d", struct.pack("<Q", u))[0]


def test_digit_split_reconstructs_within_2_to_minus_57(harness):
    rng = random.Random(11)
    rows = []
    for it in range(3000):
        k = rng.randint(1, 12)
        scale = 10.0 ** rng.randint(-300, 300) if it % 4 == 0 else 10.0 ** rng.randint(-12, 12)
        row = [rng.gauss(0, 1) * scale * 10.0 ** rng.randint(-20, 0) for _ in range(k)]
        if it % 7 == 0:
            row[0] = 0.0
        if it % 11 == 0:
            row[-1] = 5e-324 * rng.randint(1, 1 << 40)   # subnormal
        if it % 13 == 0:
            row = [0.0] * k
        rows.append(row)
    text = f"R {len(rows)}\n" + "\n".join(" ".join(f"{_bits(x):016x}" for x in r) for r in rows) + "\n"
    out = [l for l in _run(harness, text) if l]
    assert len(out) == len(rows)
    for row, line in zip(rows, out):
        v = [int(t) for t in line.split()]
        e, dig = v[0], v[1:]
        assert len(dig) == 8 * len(row)
        mx = max(abs(x) for x in row)
        if mx > 0:
            assert Fraction(2) ** (e - 1) <= Fraction(mx) < Fraction(2) ** e
        for i, x in enumerate(row):
            d = dig[8 * i:8 * i + 8]
            assert abs(d[0]) <= 128 and all(abs(m) <= 64 for m in d[1:]), d
            rec = sum(Fraction(m) * Fraction(2) ** (-7 * (p + 1)) for p, m in enumerate(d)) * Fraction(2) ** e
            assert abs(rec - Fraction(x)) <= Fraction(2) ** (e - 57), (x, e, d)


def test_level_sums_of_256_products_stay_below_2_to_24():
    # the largest digits the split can produce: |m_0| = 128, |m_p| = 64; level l holds the products
    # m_p m'_q with p + q = l, summed over K = 256 in one FP32 accumulator
    K, S = 256, 8
    bound = [128] + [64] * (S - 1)
    for lvl in range(S):
        worst = K * sum(bound[p] * bound[lvl - p] for p in range(lvl + 1))
        assert worst < 2 ** 24, (lvl, worst)


def test_single_rounding_of_the_exact_level_sum(harness):
    rng = random.Random(12)
    cases = []
    for it in range(20000):
        H = rng.randint(-(1 << 46) + 1, (1 << 46) - 1) if it % 3 else rng.randint(-50, 50)
        L = rng.randint(-(1 << 46) + 1, (1 << 46) - 1) if it % 5 else rng.randint(-(1 << 29), 1 << 29)
        if it % 7 == 0:   # cancellation: H 2^28 + L tiny
            L = max(min(-(H << 28) + rng.randint(-3000, 3000), (1 << 46) - 1), -(1 << 46) + 1)
        s = rng.randint(-140, 60) if it % 50 else rng.choice([-1150, -1100, 960, 980])
        cases.append((H, L, s))
    text = "".join(f"S {H} {L} {s}\n" for H, L, s in cases)
    out = [l for l in _run(harness, text) if l]
    assert len(out) == len(cases)
    for (H, L, s), line in zip(cases, out):
        exact = Fraction((H << 28) + L) * Fraction(2) ** s
        got = _double(int(line, 16))
        if abs(exact) >= Fraction(2) ** 1024:
            assert got == (float("inf") if exact > 0 else float("-inf")), (H, L, s, got)
        elif exact == 0 or abs(exact) >= Fraction(2) ** -1022:
            assert got == float(exact), (H, L, s, got, float(exact))   # normal range: correctly rounded
        else:
            # below the normal range the kernel rounds to 53 bits and then ldexp to the subnormal grid
            assert abs(Fraction(got) - exact) <= Fraction(2) ** -1074, (H, L, s, got)


def test_slice_products_match_exact_products_within_the_fp64_bound(harness):
    """C = A B^T formed the way the slice GEMM forms it (per-row exponents, digit slices, exact level
    sums over K <= 256, one rounding), against the exact rational products.  Per term the digit
    truncation of both operands (2^-57 of 2^e each) and the dropped levels p + q >= 8 leave at most
    2^-54 2^(e_a + e_b), with 2^e <= 2 max|row|; the final rounding adds half an ulp:
    |C - AB^T| <= K 2^-52 max|A_i| max|B_j| + 2^-53 |AB^T|."""
    rng = random.Random(13)
    for it, (m, n, k) in enumerate([(5, 4, 1), (6, 5, 7), (4, 4, 64), (3, 3, 256), (4, 2, 256)]):
        def row():
            scale = 10.0 ** rng.randint(-6, 6)
            r = [rng.gauss(0, 1) * scale * (10.0 ** rng.randint(-8, 0) if rng.random() < 0.3 else 1.0) for _ in range(k)]
            if rng.random() < 0.2:
                r[rng.randrange(k)] = 0.0
            return r
        A = [row() for _ in range(m)]
        B = [row() for _ in range(n)]
        if it == 2:   # cancellation: B's first row orthogonal-ish to A's first row
            B[0] = [-x for x in A[0]]
        text = f"G {m} {n} {k}\n" + "\n".join(" ".join(f"{_bits(x):016x}" for x in r) for r in A + B) + "\n"
        out = [l for l in _run(harness, text) if l]
        assert len(out) == m
        for i in range(m):
            vals = [_double(int(h, 16)) for h in out[i].split()]
            assert len(vals) == n
            for j in range(n):
                exact = sum(Fraction(a) * Fraction(b) for a, b in zip(A[i], B[j]))
                bound = k * Fraction(2) ** -52 * Fraction(max(abs(x) for x in A[i])) * \
                    Fraction(max(abs(x) for x in B[j])) + Fraction(2) ** -53 * abs(exact)
                assert abs(Fraction(vals[j]) - exact) <= bound, (it, i, j, vals[j], float(exact))
