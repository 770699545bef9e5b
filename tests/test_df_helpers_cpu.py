"""The integer FP64 <-> FP32 conversions and the double-float dot step of the Arnoldi kernels
(Sec. 5.1's Gram-Schmidt passes; helpers in kernels_common.cuh), compiled for the host and
checked against numpy on edge cases and seeded random values:

* f64_to_f32_trunc(v) is the binary32 value nearest v in the direction of zero (IEEE 754
  rounding toward zero) for |v| in the binary32 normal range, a signed zero below it, and a
  NaN from 2^128 up;
* split_f64(v) = (head, tail): head = f64_to_f32_trunc(v) and |head + tail - v| <= 2^-46 |v|
  (the tail keeps the top 23 of the 29 dropped fraction bits) for |v| >= 2^-80;
* f32_to_f64_bits(f) == float64(f) for every normal f, and a NaN stays a NaN;
* the double-float dot sum of 20,000 products of seeded values, against the exact sum
  (Python fractions), to 2^-40 of sum |a b|."""
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2107_04060_gb300", "csrc")
INC = os.path.join(HERE, "..", "include")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = tmp_path_factory.mktemp("dfh") / "df_host_check"
    cmd = [nvcc, "-std=c++17", "-O2", "-Xcompiler", "-ffp-contract=off", "-I", CSRC, "-I", INC,
           os.path.join(HERE, "df_host_check.cu"), "-o", str(out)]
    subprocess.run(cmd, check=True, capture_output=True, timeout=300)
    return out


def run(checker, tmp_path, v, a, b):
    inp = tmp_path / "in.f64"
    outp = tmp_path / "out.bin"
    np.concatenate([[float(len(v))], v, a, b]).astype(np.float64).tofile(inp)
    subprocess.run([str(checker), str(inp), str(outp)], check=True, timeout=60)
    raw = outp.read_bytes()
    rec = np.dtype([("t", "<f4"), ("h", "<f4"), ("l", "<f4"), ("back", "<f8")])
    per = np.frombuffer(raw[: len(v) * rec.itemsize], dtype=rec)
    sh, sl = np.frombuffer(raw[len(v) * rec.itemsize:], dtype="<f4")
    return per, sh, sl


def trunc_ref(v):
    """binary32 rounding toward zero via numpy's round-to-nearest and one step back."""
    r = np.float32(v)
    if np.isfinite(r) and abs(float(r)) > abs(v):
        r = np.nextafter(r, np.float32(0.0))
    return r


def test_conversions_and_split(checker, tmp_path):
    rng = np.random.default_rng(11)
    special = [0.0, -0.0, 1.0, -1.0, 0.1, -0.1, 1.0 / 3.0, 2.0 ** -126, -(2.0 ** -126),
               2.0 ** -127, 1e-40, 2.0 ** -80, 2.0 ** 127 * 1.9999, 2.0 ** 128, -(2.0 ** 200),
               np.inf, -np.inf, np.nan, 3.4028234e38, 1.1754944e-38, 6.02214076e23]
    randv = rng.standard_normal(3000) * 10.0 ** rng.uniform(-30, 30, 3000)
    v = np.array(special + list(randv))
    per, _, _ = run(checker, tmp_path, v, np.zeros(0), np.zeros(0))
    for k, x in enumerate(v):
        t, h, lo, back = per["t"][k], per["h"][k], per["l"][k], per["back"][k]
        ax = abs(x)
        if np.isnan(x) or ax >= 2.0 ** 128:
            assert np.isnan(t) and np.isnan(back), (x, t, back)
            continue
        if ax < 2.0 ** -126:
            assert t == 0.0 and np.signbit(t) == np.signbit(x), (x, t)
            continue
        assert t == trunc_ref(x), (x, t, trunc_ref(x))
        assert h == t
        assert back == np.float64(t)                       # f32 -> f64 exact for normals
        if ax >= 2.0 ** -80:
            err = abs(Fraction(float(h)) + Fraction(float(lo)) - Fraction(float(x)))
            assert err <= Fraction(2) ** -46 * Fraction(float(ax)), (x, h, lo)


def test_double_float_dot(checker, tmp_path):
    rng = np.random.default_rng(5)
    m = 20000
    a = rng.standard_normal(m) * 10.0 ** rng.uniform(-3, 3, m)
    b = rng.standard_normal(m)
    _, sh, sl = run(checker, tmp_path, np.zeros(0), a, b)
    exact = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b))
    scale = sum(abs(Fraction(float(x)) * Fraction(float(y))) for x, y in zip(a, b))
    got = Fraction(float(sh)) + Fraction(float(sl))
    assert abs(got - exact) <= Fraction(2) ** -40 * scale, float(abs(got - exact) / scale)
    # the FP32 product sum alone is far less accurate: the pin would catch a lost tail
    plain = float(np.sum((a.astype(np.float32) * b.astype(np.float32)).astype(np.float32)))
    assert abs(Fraction(plain) - exact) > Fraction(2) ** -40 * scale
