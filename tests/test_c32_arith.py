"""Compensated FP32 element arithmetic (csrc/c32.cuh), built for the host
from the same source and checked against exact rational arithmetic: the
split of a double into two floats, the widening back, the integer rounding
of a double to a float, the compensated dot product and reciprocal, and the
trace-form record of a triangle
(L_ij = -(a/|T|) e_i.e_j and |T|/3) within 2^-42 of the row scale, with the
range, orientation and shape cases that must fall back to FP64."""
import ctypes
import os
import shutil
import subprocess
from fractions import Fraction as Fr

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2401_15557_gb300", "csrc")


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("c32") / "libc32host.so")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-I", CSRC,
                    os.path.join(HERE, "c32_host.cpp"), "-o", out], check=True)
    L = ctypes.CDLL(out)
    fp, dp = ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_double)
    L.c32_split.argtypes = [ctypes.c_double, fp]
    L.c32_widen.argtypes = [ctypes.c_float]
    L.c32_widen.restype = ctypes.c_double
    L.c32_narrow.argtypes = [ctypes.c_double]
    L.c32_narrow.restype = ctypes.c_float
    L.c32_to_double.argtypes = [ctypes.c_float, ctypes.c_float]
    L.c32_to_double.restype = ctypes.c_double
    L.c32_two_sum.argtypes = [ctypes.c_float, ctypes.c_float, fp]
    L.c32_frcp.argtypes = [ctypes.c_float]
    L.c32_frcp.restype = ctypes.c_float
    L.c32_dot2.argtypes = [fp, fp]
    L.c32_rcp.argtypes = [ctypes.c_float, ctypes.c_float, fp]
    L.c32_tri_record.argtypes = [ctypes.c_double] * 7 + [dp]
    return L


def _split(L, x):
    hl = (ctypes.c_float * 2)()
    ok = L.c32_split(x, hl)
    return ok, float(hl[0]), float(hl[1])


def _record(L, P, a):
    o64 = (ctypes.c_double * 4)()
    ok = L.c32_tri_record(P[0][0], P[0][1], P[1][0], P[1][1], P[2][0], P[2][1], a, o64)
    return ok, np.array(o64[:])


def _exact_record(P, a):
    X = [(Fr(float(x)), Fr(float(y))) for x, y in P]
    e = [(X[(k + 2) % 3][0] - X[(k + 1) % 3][0], X[(k + 2) % 3][1] - X[(k + 1) % 3][1]) for k in range(3)]
    area2 = e[1][0] * e[2][1] - e[1][1] * e[2][0]
    nc = -2 * Fr(float(a)) / area2
    dot = lambda u, v: u[0] * v[0] + u[1] * v[1]
    L = [nc * dot(e[0], e[1]), nc * dot(e[1], e[2]), nc * dot(e[2], e[0])]
    scale = abs(nc) * max(dot(v, v) for v in e)  # the diagonal's size: the row scale
    return L, area2 / 6, scale


def test_split_is_exact_to_2m48(lib):
    rng = np.random.default_rng(1)
    xs = np.concatenate([rng.standard_normal(300) * 10.0 ** rng.integers(-11, 11, 300),
                         [1.0, -1.0, 2.0 ** -40, -(2.0 ** 40) * (1 - 2.0 ** -52), 0.3, 1 / 3]])
    for x in xs:
        ok, h, l = _split(lib, float(x))
        assert ok, x
        assert abs(Fr(float(x)) - Fr(h) - Fr(l)) <= Fr(2) ** -48 * abs(Fr(float(x))), x
        assert abs(l) < 2.0 ** -23 * abs(h)
        assert np.float32(h) == h and np.float32(l) == l
        m, _ = np.frexp(h)  # h keeps 24 significand bits: h 2^24 / 2^e is an integer
        assert float(m * 2 ** 24).is_integer()
    assert _split(lib, 0.0)[0] == 1 and _split(lib, 0.0)[1:] == (0.0, 0.0)
    assert _split(lib, -0.0)[0] == 1
    for bad in (2.0 ** -41, 2.0 ** 40, 1e300, 5e-324, float("inf"), float("nan")):
        assert _split(lib, bad)[0] == 0, bad


def test_widen_is_exact(lib):
    rng = np.random.default_rng(2)
    fs = np.concatenate([(rng.standard_normal(200) * 10.0 ** rng.integers(-30, 30, 200)).astype(np.float32),
                         np.array([0.0, -0.0, 1e-40, -1e-44, 3.4e38], dtype=np.float32)])
    sub = np.array([1e-40, -3e-42, 1.4e-45, 1.1754942e-38], dtype=np.float32)  # subnormals
    for f in np.concatenate([fs, sub, np.array([np.inf, -np.inf], dtype=np.float32)]):
        w = lib.c32_widen(float(f))
        assert w == float(f) and np.signbit(w) == np.signbit(f), f
    for bits in (0x7FC00000, 0xFFC00001, 0x7F800001, 0x7FBFFFFF):  # quiet and signalling NaNs
        assert np.isnan(lib.c32_widen(float(np.array([bits], dtype=np.uint32).view(np.float32)[0])))


def test_narrow_rounds_to_nearest_even(lib):
    rng = np.random.default_rng(6)
    xs = rng.standard_normal(2000) * 10.0 ** rng.integers(-37, 38, 2000)
    xs = xs[np.abs(xs) >= 2.0 ** -126]  # the normal floats (below them: flushed, checked at the end)
    # exact ties between two floats, both parities, and values next to them
    f = rng.standard_normal(200).astype(np.float32).astype(np.float64)
    ties = f + np.spacing(f.astype(np.float32)).astype(np.float64) / 2
    xs = np.concatenate([xs, ties, np.nextafter(ties, 0), np.nextafter(ties, np.inf), f,
                         [0.0, -0.0, 3.4028235677973366e38, 3.5e38, -1e39, float("inf"), -float("inf")]])
    with np.errstate(over="ignore"):
        for x in xs:
            n = lib.c32_narrow(float(x))
            assert np.float32(n) == np.float32(x) and np.signbit(n) == np.signbit(x), x
    assert np.isnan(lib.c32_narrow(float("nan")))
    for tiny in (1e-39, -1e-40, 5e-324):  # below the normal floats: flushed, sign kept
        n = lib.c32_narrow(tiny)
        assert n == 0.0 and np.signbit(n) == np.signbit(tiny)


def test_to_double_of_normalized_pairs(lib):
    """h + l (as TwoSum leaves it) to a double within 2^-52, including h a
    power of two with l of the other sign, zero and subnormal parts."""
    rng = np.random.default_rng(7)
    a = (rng.standard_normal(3000) * 10.0 ** rng.integers(-30, 30, 3000)).astype(np.float32)
    b = (a * rng.standard_normal(3000) * 10.0 ** rng.integers(-12, 1, 3000)).astype(np.float32)
    pw = np.float32(2.0) ** rng.integers(-60, 60, 300).astype(np.float32)
    a = np.concatenate([a, pw, -pw, np.zeros(3, np.float32), np.array([1e-40, 3e-39], np.float32)])
    b = np.concatenate([b, -pw * np.float32(1e-9), pw * np.float32(3e-8), np.array([0, 1e-41, -2e-45], np.float32),
                        np.array([1e-41, -1e-45], np.float32)])
    out = (ctypes.c_float * 2)()
    for x, y in zip(a, b):
        lib.c32_two_sum(float(x), float(y), out)
        h, l = float(out[0]), float(out[1])
        d = lib.c32_to_double(h, l)
        exact = Fr(h) + Fr(l)
        assert abs(Fr(d) - exact) <= Fr(2) ** -52 * abs(exact), (h, l, d)
        if exact == 0:
            assert d == 0.0


def test_dot2_and_rcp(lib):
    rng = np.random.default_rng(3)
    for _ in range(300):
        vals = []
        for _ in range(4):
            ok, h, l = _split(lib, float(rng.standard_normal() * 10.0 ** rng.integers(-3, 3)))
            vals += [h, l]
        # a b + c d with heavy cancellation for some draws
        if rng.random() < 0.5:
            vals[4], vals[5] = -vals[2], -vals[3]
            vals[6], vals[7] = vals[0] * (1 + 2.0 ** -20), 0.0
            vals[6] = float(np.float32(vals[6]))
        v = (ctypes.c_float * 8)(*vals)
        out = (ctypes.c_float * 2)()
        lib.c32_dot2(v, out)
        F = [Fr(x) for x in vals]
        exact = (F[0] + F[1]) * (F[2] + F[3]) + (F[4] + F[5]) * (F[6] + F[7])
        size = abs((F[0] + F[1]) * (F[2] + F[3])) + abs((F[4] + F[5]) * (F[6] + F[7]))
        assert abs(Fr(out[0]) + Fr(out[1]) - exact) <= Fr(2) ** -44 * size
        assert abs(out[1]) <= 2.0 ** -24 * abs(out[0]) or out[0] == 0.0
    for _ in range(200):
        ok, h, l = _split(lib, float(np.exp(rng.uniform(-20, 20))))
        out = (ctypes.c_float * 2)()
        lib.c32_rcp(h, l, out)
        assert abs((Fr(out[0]) + Fr(out[1])) * (Fr(h) + Fr(l)) - 1) <= Fr(5, 2) * Fr(2) ** -46
    # the float seed: within 2^-22 over the whole exponent range it is used on
    xs = np.concatenate([np.float32(2.0) ** rng.uniform(-120, 120, 4000).astype(np.float32),
                         np.float32(2.0) ** np.arange(-120, 121, dtype=np.float32),
                         np.nextafter(np.float32(2.0) ** np.arange(-120, 121, dtype=np.float32), np.float32(0))])
    for x in xs:
        r = lib.c32_frcp(float(x))
        assert abs(1 - Fr(float(x)) * Fr(r)) <= Fr(2) ** -22, x


def _jittered_triangles(rng, n, scale):
    out = []
    base = [((0.0, 0.0), (1.0, 0.0), (1.0, 1.0)), ((0.0, 0.0), (1.0, 1.0), (0.0, 1.0)),
            ((0.0, 0.0), (1.0, 0.0), (0.0, 1.0))]
    for i in range(n):
        P = np.array(base[i % 3], dtype=float)
        P += 0.2 * rng.uniform(-1, 1, (3, 2))
        off = rng.uniform(-1, 1, 2) * (1.0 if i % 2 else 0.0)
        out.append([tuple(off + scale * p) for p in P])
    return out


@pytest.mark.parametrize("scale", [1.0, 2.0 ** -10, 1e-3, 37.0])
def test_record_within_2m42_of_row_scale(lib, scale):
    rng = np.random.default_rng(int(scale * 1000) + 4)
    errs = []
    for P in _jittered_triangles(rng, 150, scale):
        sP = [(float(x), float(y)) for x, y in P]
        ax = sP[1][0] - sP[0][0], sP[1][1] - sP[0][1]
        bx = sP[2][0] - sP[0][0], sP[2][1] - sP[0][1]
        if ax[0] * bx[1] - ax[1] * bx[0] <= 0:  # keep counterclockwise ones
            sP = [sP[0], sP[2], sP[1]]
        a = float(np.exp(rng.uniform(-2, 2)))
        ok, o64 = _record(lib, sP, a)
        Lx, mT, s = _exact_record(sP, a)
        if not ok:  # only a poor angle at P0 may refuse here
            e1 = np.subtract(sP[0], sP[2])
            e2 = np.subtract(sP[1], sP[0])
            sin = abs(e1[0] * e2[1] - e1[1] * e2[0]) / (np.linalg.norm(e1) * np.linalg.norm(e2))
            assert sin < 0.26, sin
            continue
        for k in range(3):
            err = abs(Fr(float(o64[k])) - Lx[k]) / s
            errs.append(float(err))
            assert err <= Fr(2) ** -42, (k, float(err))
        assert abs(Fr(float(o64[3])) - mT) <= Fr(2) ** -42 * mT
    assert len(errs) >= 300
    assert np.median(errs) <= 2.0 ** -46, np.median(errs)


def test_record_structural_zero_and_sum(lib):
    # right angle at P0 between the axis-aligned legs e1 and e2: L12 = 0 exactly
    h = 1.0 / 1024
    ok, o64 = _record(lib, [(0.25, 0.5), (0.25 + h, 0.5), (0.25, 0.5 + h)], 1.0)
    assert ok and o64[1] == 0.0
    # e0 = (-h, h), e1 = (0, -h), e2 = (h, 0), 2|T| = h^2: L01 = L20 = -(2/h^2)(-h^2) = 2
    # exactly, and the rows of K^CR (L01 + L20 on the diagonal at P0) sum to zero
    assert o64[0] == 2.0 and o64[2] == 2.0 and abs(o64[3] - h * h / 6) <= 2.0 ** -47 * h * h / 6


def test_record_refuses_what_fp64_must_take(lib):
    ok, _ = _record(lib, [(0, 0), (0, 1), (1, 0)], 1.0)  # clockwise
    assert not ok
    # needle: the angle at P0 about 2 degrees
    ok, _ = _record(lib, [(0, 0), (1, 0), (1, 0.035)], 1.0)
    assert not ok
    # the same needle with its near-right angle at P0 is accepted, and accurate
    P = [(1.0, 0.035), (0.0, 0.0), (1.0, 0.0)]
    ok, o64 = _record(lib, P, 1.0)
    assert ok
    Lx, mT, s = _exact_record(P, 1.0)
    assert all(abs(Fr(float(o64[k])) - Lx[k]) <= Fr(2) ** -42 * s for k in range(3))
    ok, _ = _record(lib, [(0, 0), (1e-13, 0), (0, 1e-13)], 1.0)  # edges below 2^-40
    assert not ok
    for a in (2.0 ** -41, 2.0 ** 40, float("inf")):
        ok, _ = _record(lib, [(0, 0), (1, 0), (0, 1)], a)
        assert not ok, a
