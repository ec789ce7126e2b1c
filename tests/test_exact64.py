"""The exact FP64 slicing and recombination behind the FP64 tensor-core traces (csrc/exact64.h),
built for the host and checked against exact rational arithmetic (fractions.Fraction):

- the slices reproduce x truncated to a multiple of 2^-56 of the row scale, exactly, and stay
  in their digit ranges;
- the recombination of level sums is the correctly rounded FP64 value (ties to even), bit for
  bit, including ties, carries out of the mantissa, negative and zero sums;
- the fast recombination (floor(V / 2^8) rounded once) stays within its bound;
- a dot product through the slices stays within the stated error bound of the exact dot
  product, with either recombination, and its level sums stay below 2^22 (so FP32
  accumulation and the magic-number conversion are exact) up to K = 102 terms, also for the
  largest possible digits."""

import ctypes
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1502_07703_gb300", "csrc")


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    out = str(tmp_path_factory.mktemp("exact64") / "libexact64.so")
    subprocess.run([cc, "-O2", "-std=c11", "-shared", "-fPIC", "-I", CSRC, os.path.join(HERE, "exact64_shim.c"),
                    "-o", out], check=True)
    L = ctypes.CDLL(out)
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int32)
    L.shim_slices.argtypes = [dp, ctypes.c_int, ctypes.c_int, ip]
    L.shim_combine.argtypes = [ip, ctypes.c_int]
    L.shim_combine.restype = ctypes.c_double
    L.shim_combine_fast.argtypes = [ip, ctypes.c_int]
    L.shim_combine_fast.restype = ctypes.c_double
    L.shim_dot.argtypes = [dp, dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ip, ctypes.c_int]
    L.shim_dot.restype = ctypes.c_double
    return L


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _bexp(x):
    return int((np.float64(x).view(np.uint64) >> np.uint64(52)) & np.uint64(0x7FF))


def _slices(lib, x, E):
    x = np.ascontiguousarray(x, dtype=np.float64)
    a = np.zeros((len(x), 8), dtype=np.int32)
    lib.shim_slices(_ptr(x, ctypes.c_double), len(x), E, _ptr(a, ctypes.c_int32))
    return a


def test_slices_are_the_truncated_value(lib):
    rng = np.random.default_rng(11)
    xs = np.concatenate([
        rng.standard_normal(400) * np.exp2(rng.integers(-30, 30, 400)),
        [0.0, -0.0, 5e-324, -2.2e-308, 1.0, -1.0, np.nextafter(2.0, 0.0), 2.0 ** 1000, -(2.0 ** -1000)],
        [np.float64(2.0 ** 53 - 1) * 2.0 ** -52],  # all-ones mantissa: the largest top digit
    ])
    for E_extra in (0, 1, 7, 30, 70):
        E = max(_bexp(x) for x in xs) + E_extra
        if E > 2046:
            continue
        a = _slices(lib, xs, E)
        assert np.all(np.abs(a[:, 0]) <= 128) and np.all(np.abs(a[:, 1:]) <= 64)
        for x, ai in zip(xs, a):
            if _bexp(x) == 0:
                assert not ai.any(), (x, ai)
                continue
            # representation: sum_i a_i 2^(E-1029-7i)
            rep = sum(Fraction(int(ai[i])) * Fraction(2) ** (E - 1029 - 7 * i) for i in range(8))
            ulp = Fraction(2) ** (E - 1078)  # 2^-56 of the scale 2^(E-1022)
            fx = Fraction(float(x))
            trunc = (abs(fx) / ulp).__floor__() * ulp
            assert rep == (trunc if x > 0 else -trunc), (x, E)
            assert abs(rep - fx) < ulp


def _g_from_v(V):
    """Level sums G_0..G_7 with sum_s G_s 2^(7(7-s)) = V (digits of |V| in base 128, signed)."""
    s = -1 if V < 0 else 1
    m = abs(V)
    G = [0] * 8
    for k in range(7, 0, -1):
        G[k] = s * (m & 127)
        m >>= 7
    G[0] = s * m
    return G


def _combine(lib, G, Z):
    g = np.array(G, dtype=np.int32)
    return lib.shim_combine(_ptr(g, ctypes.c_int32), Z)


def _exact_float(V, Z):
    return float(Fraction(V) * Fraction(2) ** Z)  # correctly rounded, ties to even


def test_combine_is_correctly_rounded(lib):
    rng = np.random.default_rng(5)
    cases = []
    for _ in range(3000):  # random level sums within the exactness bound
        G = [int(v) for v in rng.integers(-(2 ** 22) + 1, 2 ** 22, 8)]
        cases.append((G, int(rng.integers(-900, 900))))
    for _ in range(500):  # random V, including short ones that need no rounding
        V = int(rng.integers(1, 2 ** 62)) << int(rng.integers(0, 11))
        V = V if rng.random() < 0.5 else -V
        cases.append((_g_from_v(V), int(rng.integers(-900, 900))))
    for t in range(1, 20):  # exact ties and carries out of the 53-bit mantissa
        for M in (2 ** 52, 2 ** 52 + 1, 2 ** 53 - 1, 2 ** 52 + 12345):
            for V in (M * 2 ** t + 2 ** (t - 1), M * 2 ** t + 2 ** (t - 1) - 1, M * 2 ** t + 2 ** (t - 1) + 1):
                cases.append((_g_from_v(V), -40))
                cases.append((_g_from_v(-V), 17))
    cases.append(([0] * 8, 0))
    cases.append(([1, -128, 0, 0, 0, 0, 0, 0], 3))  # cancels across levels: V = 2^49 - 2^49 = 0
    for G, Z in cases:
        V = sum(G[s] * 2 ** (7 * (7 - s)) for s in range(8))
        want = _exact_float(V, Z)
        got = _combine(lib, G, Z)
        assert np.float64(got).view(np.uint64) == np.float64(want).view(np.uint64), (G, Z, got, want)


def test_fast_combine_within_its_bound(lib):
    """floor(V / 2^8) rounded once: within 2^(Z+8) plus half an ulp of V 2^Z; exact where V is a
    multiple of 2^8 with at most 53 significant bits; zero for zero level sums."""
    rng = np.random.default_rng(6)
    cases = []
    for _ in range(3000):
        G = [int(rng.integers(-(2 ** 21) + 1, 2 ** 21))] + [int(v) for v in rng.integers(-(2 ** 22) + 1, 2 ** 22, 7)]
        cases.append((G, int(rng.integers(-900, 900))))
    for t in range(8, 30):  # small sums: few significant bits, and cancellations across levels
        cases.append((_g_from_v(3 << t), -20))
        cases.append((_g_from_v(-(5 << t)), 40))
    for G, Z in cases:
        V = sum(G[s] * 2 ** (7 * (7 - s)) for s in range(8))
        got = lib.shim_combine_fast(_ptr(np.array(G, dtype=np.int32), ctypes.c_int32), Z)
        exact = Fraction(V) * Fraction(2) ** Z
        half_ulp = Fraction(abs(got)) * Fraction(2) ** -53
        assert abs(Fraction(got) - exact) <= Fraction(2) ** (Z + 8) + half_ulp, (G, Z)
        if V % 256 == 0 and abs(V) < 2 ** 61 and (abs(V) >> 8).bit_length() <= 53:
            assert got == float(exact), (G, Z)
    assert lib.shim_combine_fast(_ptr(np.zeros(8, dtype=np.int32), ctypes.c_int32), 5) == 0.0


def _dot(lib, x, y, fast=0):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    G = np.zeros(8, dtype=np.int64)
    EF = np.zeros(2, dtype=np.int32)
    r = lib.shim_dot(_ptr(x, ctypes.c_double), _ptr(y, ctypes.c_double), len(x), _ptr(G, ctypes.c_int64),
                     _ptr(EF, ctypes.c_int32), fast)
    return r, G, int(EF[0]), int(EF[1])


@pytest.mark.parametrize("fast", [0, 1])
@pytest.mark.parametrize("K", [1, 5, 14, 30, 55, 91, 102])
def test_dot_within_bound_and_level_sums_exact_in_fp32(lib, K, fast):
    rng = np.random.default_rng(K)
    for trial in range(40):
        if trial % 4 == 0:  # modal coefficients: decaying magnitudes, mixed signs
            x = rng.standard_normal(K) * np.exp2(-np.arange(K) * 0.3)
        elif trial % 4 == 1:  # wide exponent spread
            x = rng.standard_normal(K) * np.exp2(rng.integers(-40, 3, K))
        elif trial % 4 == 2:  # cancellation: the exact sum is far below the terms
            x = rng.standard_normal(K)
        else:  # largest digits: all-ones mantissas of one sign
            x = np.full(K, (2.0 ** 53 - 1) * 2.0 ** -52)
        y = rng.standard_normal(K) * 3.0 if trial % 4 != 3 else np.full(K, -(2.0 ** 53 - 1) * 2.0 ** -50)
        if trial % 4 == 2 and K > 1:
            y[-1] = 0.0
            y[-1] = -float(np.dot(x[:-1], y[:-1])) / x[-1]
        r, G, E, F = _dot(lib, x, y, fast)
        bounds = [K * 16384] + [K * 4096 * (s + 3) for s in range(1, 8)]
        assert all(abs(int(G[s])) <= bounds[s] for s in range(8)), (G, bounds)
        assert np.all(np.abs(G) < 2 ** 22)
        exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(x, y))
        scale = Fraction(2) ** (E + F - 2044)
        half_ulp = Fraction(abs(r)) * Fraction(2) ** -53 if r != 0 else 0
        # inputs truncated (2 K 2^-56), levels 8..14 dropped (7.1 K 2^-58), the fast form's
        # floor (2^-55, of the scale 2^(E+F-2044)), the final rounding
        bound = (Fraction(151, 10) * K * Fraction(2) ** -58 + fast * Fraction(2) ** -55) * scale + half_ulp
        assert abs(Fraction(r) - exact) <= bound, (K, trial, float(abs(Fraction(r) - exact) / scale))
