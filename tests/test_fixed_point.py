"""CPU tests of the integer digit arithmetic that the complex128 tensor-core kernel uses
(fixed_point.h): the split of a double into six 9-bit digits, the rounding of a 64-bit
integer times a power of two to the nearest double, and one group's contraction with
exact level sums, each against exact rational arithmetic."""
import ctypes
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fx(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("fx") / "libfxh.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC",
                    os.path.join(ROOT, "tests", "fixed_point_harness.cpp"), "-o", out], check=True)
    lib = ctypes.CDLL(out)
    lib.fx_to_fixed.restype = ctypes.c_longlong
    lib.fx_to_fixed.argtypes = [ctypes.c_double, ctypes.c_uint]
    lib.fx_exp_field.restype = ctypes.c_uint
    lib.fx_exp_field.argtypes = [ctypes.c_double]
    lib.fx_digits.argtypes = [ctypes.c_longlong, ctypes.POINTER(ctypes.c_int)]
    lib.fx_assemble.restype = ctypes.c_double
    lib.fx_assemble.argtypes = [ctypes.c_longlong, ctypes.c_int]
    dp = ctypes.POINTER(ctypes.c_double)
    lib.fx_group_apply.argtypes = [dp, dp, dp, ctypes.POINTER(ctypes.c_longlong)]
    lib.fx_assemble_words.restype = ctypes.c_double
    lib.fx_assemble_words.argtypes = [ctypes.c_longlong, ctypes.c_int]
    lib.fx_small_float_to_int.restype = ctypes.c_int
    lib.fx_small_float_to_int.argtypes = [ctypes.c_float]
    lib.fx_combine_words.restype = ctypes.c_double
    lib.fx_combine_words.argtypes = [ctypes.c_int] * 5 + [ctypes.c_int]
    lib.fx_digit_pair_words.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_uint,
                                        ctypes.POINTER(ctypes.c_uint)]
    return lib


def _round_half_away(q: Fraction) -> int:
    f = q.numerator // q.denominator
    r = q - f
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and q > 0):
        return f + 1
    return f


def _digits(fx, x):
    d = (ctypes.c_int * 6)()
    fx.fx_digits(x, d)
    return list(d)


def test_split_is_exact_rounding_and_digits_reconstruct(fx):
    rng = np.random.default_rng(7)
    xs = list(rng.standard_normal(300) * np.exp2(rng.integers(-60, 60, 300)))
    xs += [0.0, -0.0, 1.0, -1.0, 2.0 ** -1074, 5e-324 * 7, np.nextafter(2.0, 0.0), -np.nextafter(1.0, 0.0)]
    for x in xs:
        x = float(x)
        emax_own = fx.fx_exp_field(x)
        for emax in (emax_own, emax_own + 1, emax_own + 13, emax_own + 60):
            e = emax - 1022
            X = fx.fx_to_fixed(x, emax)
            assert X == _round_half_away(Fraction(x) * Fraction(2) ** (53 - e)), (x, emax)
            assert abs(X) < 2 ** 53
            d = _digits(fx, X)
            assert -256 <= d[0] <= 256 and all(-256 <= v <= 255 for v in d[1:])
            assert sum(v * 2 ** (9 * (5 - i)) for i, v in enumerate(d)) == X


def test_digit_extremes(fx):
    for X in (2 ** 53 - 1, -(2 ** 53 - 1), 0, 1, -1, 255, 256, -256, 2 ** 45 * 256 - 1):
        d = _digits(fx, X)
        assert -256 <= d[0] <= 256 and all(-256 <= v <= 255 for v in d[1:])
        assert sum(v * 2 ** (9 * (5 - i)) for i, v in enumerate(d)) == X


def _nearest(z: int, p: int) -> float:
    # Python's int / int true division rounds correctly (ties to even)
    return float(z * 2 ** p) if p >= 0 else z / 2 ** (-p)


def test_assemble_rounds_to_nearest_even(fx):
    rng = np.random.default_rng(8)
    cases = []
    for _ in range(2000):
        bits = int(rng.integers(0, 62))
        z = int(rng.integers(1, 2 ** 62)) >> (61 - bits)
        z = z if rng.random() < 0.5 else -z
        cases.append((z, int(rng.integers(-1000, 900))))
    # exact ties and carries into the next binade
    for t in range(53, 62):
        r = t - 52
        base = 1 << t
        cases += [(base + (1 << (r - 1)), -40), (base + 3 * (1 << (r - 1)), -40),
                  ((1 << (t + 1)) - 1, -40), (-((1 << (t + 1)) - (1 << (r - 1))), 7)]
    for z, p in cases:
        if z == 0:
            continue
        assert fx.fx_assemble(z, p) == _nearest(z, p), (z, p)
    assert fx.fx_assemble(0, -5) == 0.0


def test_assemble_subnormal_within_one_ulp(fx):
    for z, p in ((3, -1080), (2 ** 40 + 12345, -1100), (-(2 ** 61 - 1), -1130)):
        got, want = fx.fx_assemble(z, p), _nearest(z, p)
        assert abs(got - want) <= 5e-324 * 1.0000001


def _group(fx, a, u):
    a = np.ascontiguousarray(np.stack([a.real, a.imag], -1).reshape(-1), dtype=np.float64)
    u = np.ascontiguousarray(np.stack([u.real, u.imag], -1).reshape(-1), dtype=np.float64)
    out = np.zeros(32)
    lmax = (ctypes.c_longlong * 6)()
    dp = ctypes.POINTER(ctypes.c_double)
    fx.fx_group_apply(a.ctypes.data_as(dp), u.ctypes.data_as(dp), out.ctypes.data_as(dp), lmax)
    return out[0::2] + 1j * out[1::2], list(lmax)


def _check_group(fx, a, u):
    got, lmax = _group(fx, a, u)
    # FP32 accumulation is exact for the levels kept in their own accumulators
    assert max(lmax[:5]) <= 2 ** 24
    comps = np.concatenate([a.real, a.imag])
    ea = int(np.frexp(np.max(np.abs(comps)))[1]) if np.any(comps) else -1021
    ub = np.concatenate([u.real.ravel(), u.imag.ravel()])
    eb = int(np.frexp(np.max(np.abs(ub)))[1])
    bound_scale = Fraction(2) ** (ea + eb - 46)
    for n in range(16):
        re = sum(Fraction(float(u[n, l].real)) * Fraction(float(a[l].real)) -
                 Fraction(float(u[n, l].imag)) * Fraction(float(a[l].imag)) for l in range(16))
        im = sum(Fraction(float(u[n, l].real)) * Fraction(float(a[l].imag)) +
                 Fraction(float(u[n, l].imag)) * Fraction(float(a[l].real)) for l in range(16))
        for exact, g in ((re, got[n].real), (im, got[n].imag)):
            half_ulp = Fraction(float(np.spacing(abs(float(exact))))) / 2
            assert abs(Fraction(float(g)) - exact) <= bound_scale + half_ulp, (n, float(exact), g)


def test_group_contraction_within_bound(fx):
    rng = np.random.default_rng(9)
    for trial in range(12):
        u = np.array(W.haar_unitary(16, rng), dtype=np.complex128).reshape(16, 16)
        a = rng.standard_normal(16) + 1j * rng.standard_normal(16)
        if trial % 3 == 1:
            a *= np.exp2(rng.integers(-40, 1, 16))          # mixed magnitudes in one row
        if trial % 3 == 2:
            a[rng.integers(0, 16, 5)] = 0.0                    # zeros
            a *= 1e-150
        _check_group(fx, a, u)


def test_group_contraction_non_unitary_and_large_entries(fx):
    rng = np.random.default_rng(10)
    u = (rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16))) * 37.5
    a = rng.standard_normal(16) + 1j * rng.standard_normal(16)
    _check_group(fx, a, u)
    # a matrix whose every entry and every amplitude sits at the top of its digit range
    u = np.full((16, 16), (1 - 2 ** -53) * (1 + 1j))
    a = np.full(16, -(1 - 2 ** -53) * (1 - 1j))
    _check_group(fx, a, u)


def test_identity_and_permutation_return_input_exactly(fx):
    # amplitudes on the row's fixed-point grid (2^-52 below a largest component in [1, 2))
    # come back bit for bit; off-grid bits below 2^-53 of the largest are rounded away
    rng = np.random.default_rng(11)
    a = (rng.integers(-2 ** 40, 2 ** 40, 16) + 1j * rng.integers(-2 ** 40, 2 ** 40, 16)) / 2.0 ** 40
    a[3] = 1.75 - 1j
    got, _ = _group(fx, a, np.eye(16, dtype=np.complex128))
    assert np.array_equal(got, a)
    perm = rng.permutation(16)
    P = np.eye(16, dtype=np.complex128)[perm]
    got, _ = _group(fx, a, P)
    assert np.array_equal(got, a[perm])
    got, _ = _group(fx, np.zeros(16, dtype=np.complex128), P)
    assert np.array_equal(got, np.zeros(16))


def test_kernel_digit_words_match_reference_split(fx):
    """The kernel's 32-bit-word split gives the reference digits, packed as FP16 patterns
    of 2048 + 2u whose (x 0.5 - 1280) is the digit."""
    rng = np.random.default_rng(12)
    vals = list(rng.standard_normal(400) * np.exp2(rng.integers(-70, 10, 400)))
    vals += [0.0, -0.0, 5e-324, -3e-320, 1.5, -1.5, np.nextafter(1.0, 2.0), -(2.0 - 2 ** -52)]
    w = (ctypes.c_uint * 6)()
    for trial in range(600):
        re, im = float(rng.choice(vals)), float(rng.choice(vals))
        emax = max(fx.fx_exp_field(re), fx.fx_exp_field(im)) + int(rng.choice([0, 0, 1, 5, 31, 32, 33, 53, 54, 70]))
        fx.fx_digit_pair_words(re, im, emax, w)
        dr = _digits(fx, fx.fx_to_fixed(re, emax))
        di = _digits(fx, fx.fx_to_fixed(im, emax))
        for i in range(6):
            lo, hi = w[i] & 0xFFFF, w[i] >> 16
            for half, want in ((lo, dr[i]), (hi, di[i])):
                assert half & 0xFC00 == 0x6800, hex(w[i])
                h = np.array([half], dtype=np.uint16).view(np.float16).astype(np.float64)[0]
                assert h * 0.5 - 1280.0 == want, (re, im, emax, i)


def test_assemble_words_equals_assemble(fx):
    rng = np.random.default_rng(13)
    for _ in range(4000):
        bits = int(rng.integers(0, 63))
        z = int(rng.integers(0, 2 ** 62)) >> (62 - bits)
        z = z if rng.random() < 0.5 else -z
        p = int(rng.integers(-1200, 1000))
        a, b = fx.fx_assemble(z, p), fx.fx_assemble_words(z, p)
        assert (a == b and np.signbit(a) == np.signbit(b)) or (np.isnan(a) and np.isnan(b)), (z, p)
    for z in (1, -1, 2 ** 32, 2 ** 32 - 1, -(2 ** 32), 2 ** 61 + 2 ** 8 + 1, 2 ** 53 + 1, 0):
        assert fx.fx_assemble_words(z, -60) == fx.fx_assemble(z, -60)


def test_small_float_to_int_range(fx):
    rng = np.random.default_rng(14)
    ints = [0, 1, -1, 2 ** 22, -(2 ** 22), 2 ** 22 - 1, -(2 ** 22) + 1] + \
        list(rng.integers(-(2 ** 22), 2 ** 22 + 1, 2000))
    for v in ints:
        assert fx.fx_small_float_to_int(float(v)) == int(v)


def test_combine_words_matches_exact(fx):
    rng = np.random.default_rng(15)
    for _ in range(2000):
        i0, i1 = (int(x) for x in rng.integers(-(2 ** 21), 2 ** 21 + 1, 2))
        i2, i3 = (int(x) for x in rng.integers(-(2 ** 23), 2 ** 23 + 1, 2))
        i45 = int(rng.integers(-(2 ** 27), 2 ** 27))
        p = int(rng.integers(-1100, -40))
        z = i0 * 2 ** 40 + i1 * 2 ** 31 + i2 * 2 ** 22 + i3 * 2 ** 13 + i45
        got = fx.fx_combine_words(i0, i1, i2, i3, i45, p)
        if z == 0:
            assert got == 0.0
        elif abs(_nearest(z, p)) >= 2.0 ** -1022:
            assert got == _nearest(z, p)
