"""Host pins of the digit form of the dense solve (csrc/emt_digits.cuh).

The forward kernel computes v = X i as an exact integer product of base-256
digits on the bf16 tensor cores and rounds the result once to double.  The
integer helpers it uses are compiled here for the CPU and checked against
exact rational arithmetic (fractions.Fraction):

* the 62-bit fixed-point rounding of a double against a shared scale,
* the balanced digits (their sum reconstructs the integer; each fits bf16),
* the rounding of the 128-bit group sum T to double (correct rounding),
* a whole row product emulated with exact integer digit products, grouped
  and truncated as the kernel does, against the exact dot product.
"""
import ctypes
import os
import random
import struct
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HDR = os.path.join(os.path.dirname(HERE), "paper_1903_01081_b300", "csrc", "emt_digits.cuh")

SHIM = r"""
#include "%s"
using namespace emt;
extern "C" {
long long t_fixed(double x, unsigned emax) { return dg_fixed(x, emax); }
int t_digit(long long n, int j) { return dg_digit(n + kDigitBias, j); }
unsigned t_digit_bf16(long long n, int j) { return dg_digit_bf16(n + kDigitBias, j); }
double t_to_double(long long ta, long long tb, int xexp) { return dg_to_double(ta, tb, xexp); }
int t_acc_int(float d) { return dg_acc_int(d); }
// one row of v = X i the way the kernel does it, with exact integer digit products
double t_dot(const double* x, const double* iv, int K) {
  unsigned er = 1, ei = 1;
  for (int k = 0; k < K; ++k) { if (dg_expo(x[k]) > er) er = dg_expo(x[k]); if (dg_expo(iv[k]) > ei) ei = dg_expo(iv[k]); }
  long long g[2 * kDigits] = {0};
  for (int k = 0; k < K; ++k) {
    const long long m = dg_fixed(x[k], er) + kDigitBias, n = dg_fixed(iv[k], ei) + kDigitBias;
    for (int a = 0; a < kDigits; ++a)
      for (int b = 0; b < kDigits; ++b) g[a + b] += (long long)dg_digit(m, a) * dg_digit(n, b);
  }
  long long ta = 0, tb = 0;
  for (int s = kDigitGroupLo; s < 2 * kDigits - 1; ++s) {
    if (s >= 11) ta += (long long)((unsigned long long)g[s] << (8 * (s - 11)));
    else tb += (long long)((unsigned long long)g[s] << (8 * (s - kDigitGroupLo)));
  }
  return dg_to_double(ta, tb, (int)er + (int)ei - 2120);
}
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    d = tmp_path_factory.mktemp("digits")
    src = d / "shim.cpp"
    src.write_text(SHIM % HDR)
    so = d / "libshim.so"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", str(so), str(src)])
    L = ctypes.CDLL(str(so))
    L.t_fixed.restype = ctypes.c_longlong
    L.t_fixed.argtypes = [ctypes.c_double, ctypes.c_uint]
    L.t_digit.restype = ctypes.c_int
    L.t_digit.argtypes = [ctypes.c_longlong, ctypes.c_int]
    L.t_digit_bf16.restype = ctypes.c_uint
    L.t_digit_bf16.argtypes = [ctypes.c_longlong, ctypes.c_int]
    L.t_to_double.restype = ctypes.c_double
    L.t_to_double.argtypes = [ctypes.c_longlong, ctypes.c_longlong, ctypes.c_int]
    L.t_acc_int.restype = ctypes.c_int
    L.t_acc_int.argtypes = [ctypes.c_float]
    L.t_dot.restype = ctypes.c_double
    L.t_dot.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), ctypes.c_int]
    return L


def expo(x: float) -> int:
    return (struct.unpack("<Q", struct.pack("<d", x))[0] >> 52) & 0x7FF


def round_half_away(q: Fraction) -> int:
    f = abs(q)
    n = int(f)
    if f - n >= Fraction(1, 2):
        n += 1
    return n if q >= 0 else -n


def test_fixed_point_rounding_is_exact(lib):
    rng = random.Random(1)
    for _ in range(4000):
        x = rng.uniform(-1, 1) * 2.0 ** rng.randint(-60, 60)
        emax = expo(x) + rng.choice([0, 0, 1, 5, 30, 53, 70])
        want = round_half_away(Fraction(x) * Fraction(2) ** (62 - (emax - 1022)))
        got = lib.t_fixed(x, emax)
        assert got == want, (x, emax)
        assert abs(got) <= 2 ** 62
    assert lib.t_fixed(0.0, 1000) == 0 and lib.t_fixed(5e-324, 1000) == 0   # zero and subnormal


def test_balanced_digits_reconstruct_and_fit_bf16(lib):
    rng = random.Random(2)
    vals = [0, 1, -1, 2 ** 62 - 1, -(2 ** 62) + 1, 2 ** 62, -(2 ** 62), 0x7F7F7F7F7F7F7F, -0x8080808080808]
    vals += [rng.randint(-(2 ** 62), 2 ** 62) for _ in range(3000)]
    for n in vals:
        d = [lib.t_digit(n, j) for j in range(8)]
        assert sum(dj * 256 ** j for j, dj in enumerate(d)) == n
        assert all(-128 <= dj <= 127 for dj in d[:7]) and -65 <= d[7] <= 64
        for j, dj in enumerate(d):
            bits = struct.unpack("<I", struct.pack("<f", float(dj)))[0]
            assert bits & 0xFFFF == 0                      # 8 significant bits at most: exact in bf16
            assert lib.t_digit_bf16(n, j) == bits >> 16


def test_accumulator_to_int_is_exact(lib):
    for v in [0, 1, -1, 4161600, -4161600, 2 ** 21, -(2 ** 21), 2 ** 22 - 1, -(2 ** 22) + 1, 123457, -99999]:
        assert lib.t_acc_int(float(v)) == v


def test_group_sum_rounds_once_to_nearest_even(lib):
    rng = random.Random(3)
    cases = [(0, 0, 0), (0, 1, 0), (0, -1, 5), (1, 0, -40), (-1, 0, -40), (2 ** 47, 2 ** 55, -1100),
             (-(2 ** 47), -(2 ** 55), 7), (0, (1 << 53) + 1, 0), (0, (1 << 54) + 2, 0), (0, (1 << 54) + 6, 0)]
    for _ in range(5000):
        cases.append((rng.randint(-(2 ** 48), 2 ** 48), rng.randint(-(2 ** 56), 2 ** 56), rng.randint(-1150, 900)))
    for _ in range(2000):   # ties and near-ties of the 53-bit rounding
        m = rng.randint(2 ** 52, 2 ** 53 - 1)
        sh = rng.randint(1, 30)
        t = (m << sh) + rng.choice([0, 1, -1]) + (1 << (sh - 1)) * rng.choice([0, 1])
        cases.append((t >> 40, t & ((1 << 40) - 1), rng.randint(-200, 200)))
    for ta, tb, xe in cases:
        exact = Fraction(ta * 2 ** 40 + tb) * Fraction(2) ** xe
        want = float(exact)   # Python rounds a Fraction correctly (nearest, ties to even)
        if want != 0.0 and abs(want) < 2.0 ** -1022:
            want = 0.0        # below the normal range the kernel flushes to zero
        assert lib.t_to_double(ta, tb, xe) == want, (ta, tb, xe)


def test_row_product_against_the_exact_dot_product(lib):
    """Error of the emulated digit product: at most one rounding of the exact
    result plus 2^-60 of sum_k max|X| max|i| (the two fixed-point roundings
    and the dropped digit pairs)."""
    rng = np.random.default_rng(4)
    for trial in range(400):
        K = int(rng.integers(1, 129))
        x = rng.standard_normal(K) * np.exp(rng.uniform(-12, 12, K))
        iv = rng.standard_normal(K) * np.exp(rng.uniform(-8, 8, K))
        if trial % 7 == 0:
            x[rng.integers(0, K)] = 0.0
        got = lib.t_dot(x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                        iv.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), K)
        exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(x, iv))
        scale = K * float(np.max(np.abs(x))) * float(np.max(np.abs(iv)))
        err = abs(Fraction(got) - exact)
        bound = Fraction(abs(float(exact))) * Fraction(2) ** -53 + Fraction(scale) * Fraction(2) ** -60
        assert err <= bound, (trial, float(err), float(bound))


def test_cancelling_row_product_keeps_absolute_accuracy(lib):
    """Two nearly equal large products of opposite sign (the strong-branch
    case): the digit product is exact up to the fixed-point roundings, so the
    small difference keeps an absolute error of ~2^-62 of the large terms."""
    x = np.array([1.0, 1.0 - 2.0 ** -40, 3e-9])
    iv = np.array([1e4, -1e4, 1.0])
    got = lib.t_dot(x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                    iv.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 3)
    exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(x, iv))
    assert abs(Fraction(got) - exact) <= Fraction(1e4) * Fraction(2) ** -60
