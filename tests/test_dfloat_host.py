"""The double-float arithmetic of the refinement residual, pinned on the CPU.

`csrc/elas_dfloat.cuh` holds the operations the double-float kernels use: Knuth's TwoSum,
Dekker's Fast2Sum, the FMA-based exact product, the unnormalised double-word sum, product
and multiply-add analysed by Joldes, Muller and Popescu (ACM TOMS 44, 2017), and the
bit-level conversions between FP64 values and FP32 pairs.  The same source compiles for
the host (binary32 and binary64, round to nearest, no contraction); the driver
`tests/dfloat_host_check.cu` applies one operation to seeded inputs, and these tests check
every output against exact rational arithmetic:

* TwoSum and Fast2Sum are error-free: s = fl(a + b) and s + e = a + b exactly.
* The double-word sum, products and multiply-add stay within a few 2^-47 of the
  operands' magnitudes; a 27-term stencil row accumulated by multiply-adds stays within
  2^-40 of the sum of |a_i b_i| (an FP32 evaluation errs by about 2^-24).
* The FP64 -> pair split keeps exactly the leading 47 significant bits (24 in hi, 23 in
  lo), 24 bits below 2^-103 and nothing below 2^-126; the FP32 -> FP64 conversion is
  exact for normal values and gives 0 for subnormals.
"""
import os
import shutil
import struct
import subprocess
from fractions import Fraction as Fr

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "dfloat_host_check.cu")
P47 = Fr(1, 2 ** 47)


@pytest.fixture(scope="module")
def run(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("no nvcc")
    d = tmp_path_factory.mktemp("dfloat")
    exe = str(d / "dfloat_host_check")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-ffp-contract=off",
                    "-gencode", "arch=compute_103a,code=sm_103a", SRC, "-o", exe], check=True)

    def call(op, records, out_dtype, out_width):
        records = np.ascontiguousarray(records)
        fin, fout = str(d / f"{op}.in"), str(d / f"{op}.out")
        records.tofile(fin)
        n = records.shape[0]
        subprocess.run([exe, op, str(n), fin, fout], check=True)
        out = np.fromfile(fout, dtype=out_dtype)
        return out.reshape(n, out_width) if out_width > 1 else out

    return call


def f32_values(rng, n, lo_exp=-20, hi_exp=20):
    """Random FP32 values of random sign with exponents spread over [lo_exp, hi_exp]."""
    mant = rng.uniform(1.0, 2.0, n)
    return (mant * 2.0 ** rng.integers(lo_exp, hi_exp + 1, n) * rng.choice([-1.0, 1.0], n)).astype(np.float32)


def pairs(rng, n, lo_rel=2.0 ** -24):
    """Double-float pairs (hi, lo) with |lo| <= lo_rel |hi|, as the kernels' splits give."""
    hi = f32_values(rng, n)
    lo = (hi.astype(np.float64) * rng.uniform(-lo_rel, lo_rel, n)).astype(np.float32)
    return hi, lo


def F(x):
    return Fr(float(x))      # exact: every binary32 / binary64 value is a rational


def mag(hi, lo):
    return abs(F(hi)) + abs(F(lo))


def test_two_sum_and_fast_two_sum_are_error_free(run):
    rng = np.random.default_rng(1)
    n = 6000
    a = f32_values(rng, n)
    b = f32_values(rng, n)
    b[: n // 4] = -a[: n // 4] * np.float32(1 + 2.0 ** -20)     # near-cancelling pairs
    b[n // 4: n // 2] = (a[n // 4: n // 2] * 2.0 ** -30).astype(np.float32)   # far apart
    out = run("two_sum", np.stack([a, b], 1), np.float32, 2)
    assert np.array_equal(out[:, 0], a + b)                    # s = fl(a + b) (numpy FP32 adds round to nearest)
    for (x, y), (s, e) in zip(zip(a, b), out):
        assert F(s) + F(e) == F(x) + F(y)
    big = np.where(np.abs(a) >= np.abs(b), a, b)
    small = np.where(np.abs(a) >= np.abs(b), b, a)
    out = run("fast_sum", np.stack([big, small], 1), np.float32, 2)
    for (x, y), (s, e) in zip(zip(big, small), out):
        assert F(s) + F(e) == F(x) + F(y)


def test_pair_sum_within_a_few_2_47_of_the_operands(run):
    rng = np.random.default_rng(2)
    n = 6000
    xh, xl = pairs(rng, n)
    yh, yl = pairs(rng, n)
    yh[: n // 3], yl[: n // 3] = -xh[: n // 3], (-xl[: n // 3] * np.float32(0.75))   # cancellation
    out = run("add", np.stack([xh, xl, yh, yl], 1), np.float32, 2)
    worst = Fr(0)
    for i in range(n):
        exact = F(xh[i]) + F(xl[i]) + F(yh[i]) + F(yl[i])
        scale = mag(xh[i], xl[i]) + mag(yh[i], yl[i])
        err = abs(F(out[i, 0]) + F(out[i, 1]) - exact)
        assert err <= 2 * P47 * scale, i
        assert abs(F(out[i, 1])) <= Fr(1, 2 ** 22) * scale         # lo stays a few 2^-24 of the operands
        worst = max(worst, err / scale)
    assert worst > 0                                                # the bound is not vacuous


def test_pair_products_within_a_few_2_47_of_the_operands(run):
    rng = np.random.default_rng(3)
    n = 6000
    xh, xl = pairs(rng, n)
    yh, yl = pairs(rng, n)
    out = run("mul", np.stack([xh, xl, yh, yl], 1), np.float32, 2)
    for i in range(n):
        exact = (F(xh[i]) + F(xl[i])) * (F(yh[i]) + F(yl[i]))
        err = abs(F(out[i, 0]) + F(out[i, 1]) - exact)
        assert err <= 3 * P47 * mag(xh[i], xl[i]) * mag(yh[i], yl[i]), i
    y = f32_values(rng, n)
    out = run("mulf", np.stack([xh, xl, y], 1), np.float32, 2)
    for i in range(n):
        exact = (F(xh[i]) + F(xl[i])) * F(y[i])
        err = abs(F(out[i, 0]) + F(out[i, 1]) - exact)
        assert err <= 2 * P47 * mag(xh[i], xl[i]) * abs(F(y[i])), i


def test_pair_multiply_add_within_a_few_2_47_of_the_operands(run):
    rng = np.random.default_rng(4)
    n = 6000
    ah, al = pairs(rng, n)
    bh, bl = pairs(rng, n)
    ch, cl = pairs(rng, n)
    k = n // 3                                    # c cancelling a b
    prod = (ah[:k].astype(np.float64) * bh[:k].astype(np.float64))
    ch[:k] = (-prod).astype(np.float32)
    cl[:k] = (-(prod + ch[:k].astype(np.float64))).astype(np.float32)
    out = run("fma", np.stack([ah, al, bh, bl, ch, cl], 1), np.float32, 2)
    for i in range(n):
        exact = (F(ah[i]) + F(al[i])) * (F(bh[i]) + F(bl[i])) + F(ch[i]) + F(cl[i])
        scale = mag(ah[i], al[i]) * mag(bh[i], bl[i]) + mag(ch[i], cl[i])
        err = abs(F(out[i, 0]) + F(out[i, 1]) - exact)
        assert err <= 6 * P47 * scale, i


def test_stencil_row_of_27_multiply_adds(run):
    """A 27-term row (one node's neighbourhood) accumulated without renormalisation:
    within 2^-40 of sum |a_i b_i|, where an FP32 evaluation errs by about 2^-24."""
    rng = np.random.default_rng(5)
    n = 400
    ah, al = pairs(rng, 27 * n)
    bh, bl = pairs(rng, 27 * n)
    a = np.stack([ah, al], 1).reshape(n, 54)
    b = np.stack([bh, bl], 1).reshape(n, 54)
    out = run("dot27", np.concatenate([a, b], 1), np.float32, 2)
    worst32 = 0.0
    for i in range(n):
        ta = [F(a[i, 2 * k]) + F(a[i, 2 * k + 1]) for k in range(27)]
        tb = [F(b[i, 2 * k]) + F(b[i, 2 * k + 1]) for k in range(27)]
        exact = sum(x * y for x, y in zip(ta, tb))
        scale = sum(abs(x * y) for x, y in zip(ta, tb))
        err = abs(F(out[i, 0]) + F(out[i, 1]) - exact)
        assert err <= Fr(1, 2 ** 40) * scale, i
        s32 = np.float32(0)
        for k in range(27):
            s32 = np.float32(s32 + np.float32(a[i, 2 * k]) * np.float32(b[i, 2 * k]))
        worst32 = max(worst32, float(abs(F(s32) - exact) / scale))
    assert worst32 > 2.0 ** -30           # the FP32 evaluation of the same rows is far coarser


def test_pair_to_float_rounds_once(run):
    rng = np.random.default_rng(6)
    n = 6000
    hi = f32_values(rng, n)
    lo = (hi.astype(np.float64) * rng.uniform(2.0 ** -28, 2.0 ** -23, n) * rng.choice([-1.0, 1.0], n)).astype(np.float32)
    out = run("to_float", np.stack([hi, lo], 1), np.float32, 1)
    # hi + lo is exact in FP64 here (|lo| >= 2^-28 |hi|), so one FP32 rounding of it is the reference
    assert np.array_equal(out, (hi.astype(np.float64) + lo.astype(np.float64)).astype(np.float32))


def truncated(v, bits):
    """v with its significand truncated to `bits` significant bits (exact)."""
    b = struct.unpack("<Q", struct.pack("<d", v))[0]
    e = (b >> 52) & 0x7FF
    m = (b & ((1 << 52) - 1)) | (1 << 52)
    m = (m >> (53 - bits)) << (53 - bits)
    return (-1 if b >> 63 else 1) * Fr(m) * Fr(2) ** (e - 1075)


def test_split_keeps_the_leading_47_bits(run):
    rng = np.random.default_rng(7)
    n = 6000
    v = rng.uniform(1.0, 2.0, n) * 2.0 ** rng.integers(-140, 127, n) * rng.choice([-1.0, 1.0], n)
    edges = [2.0 ** -126, np.nextafter(2.0 ** -126, 0), 2.0 ** -103, np.nextafter(2.0 ** -103, 0),
             1.0, -1.0, np.nextafter(2.0 ** 128, 0), -np.nextafter(2.0 ** 128, 0), 0.0, -0.0, 5e-324,
             1.0 + 2.0 ** -52, 1.0 + 2.0 ** -46, 1.0 + 2.0 ** -47, 1.0 / 3.0, -np.pi * 1e-9]
    v = np.concatenate([v, np.array(edges)])
    out = run("split", v, np.float32, 2)
    for x, (hi, lo) in zip(v, out):
        x = float(x)
        e = (struct.unpack("<Q", struct.pack("<d", x))[0] >> 52) & 0x7FF
        if e < 897:                              # below 2^-126: (0, 0)
            assert hi == 0 and lo == 0, x
            continue
        assert F(hi) == truncated(x, 24), x      # hi: the leading 24 bits
        keep = 47 if e >= 920 else 24            # lo: the next 23 bits, from 2^-103 up
        assert F(hi) + F(lo) == truncated(x, keep), x
        assert abs(F(x) - F(hi) - F(lo)) < Fr(2) ** -46 * abs(F(x)) or keep == 24


def test_constant_constructor_and_float_to_double(run):
    rng = np.random.default_rng(8)
    n = 6000
    v = rng.uniform(1.0, 2.0, n) * 2.0 ** rng.integers(-60, 60, n) * rng.choice([-1.0, 1.0], n)
    out = run("ctor", v, np.float32, 2)
    for x, (hi, lo) in zip(v, out):
        assert hi == np.float32(x)                                   # hi = RN(v)
        assert abs(F(x) - F(hi) - F(lo)) <= Fr(1, 2 ** 48) * abs(F(x))
    x = f32_values(rng, n, -126, 127)
    sub = np.array([1e-45, -1e-40, 0.0, -0.0, np.finfo(np.float32).tiny, -np.finfo(np.float32).max],
                   dtype=np.float32)
    x = np.concatenate([x, sub])
    out = run("f2d", x, np.float64, 1)
    normal = np.abs(x) >= np.finfo(np.float32).tiny
    assert np.array_equal(out[normal], x[normal].astype(np.float64))   # exact
    assert np.all(out[~normal] == 0.0)                                 # subnormals and zeros
