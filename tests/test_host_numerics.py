"""Host checks of numerical building blocks of the CUDA path, compiled from
the library's own headers with nvcc (host code; no GPU needed):
- two_sum is error-free: s + e equals a + b exactly;
- double-float addition and multiplication are accurate to ~2^-44 relative
  to the operands, and a long double-float accumulation matches the exact sum;
- spd_inv3 (the coarse block-Jacobi inverse) returns the inverse of a
  well-conditioned SPD block and a symmetric positive definite block with
  bounded eigenvalues for nearly singular, indefinite or zero blocks.
References are exact rational arithmetic and numpy eigenvalues."""
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    if not shutil.which(NVCC) and not os.path.exists(NVCC):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("hn") / "host_numerics")
    cmd = [NVCC, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
           "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "host_numerics.cu"), "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True, timeout=600)
    return exe


def run(exe, lines):
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True,
                         timeout=120).stdout
    return [[float.fromhex(t) for t in ln.split()] for ln in out.strip().splitlines()]


def f32(x):
    return float(np.float32(x))


def test_two_sum_is_error_free(driver):
    rng = np.random.default_rng(1)
    pairs = []
    for _ in range(3000):
        a = f32(rng.standard_normal() * 10.0 ** rng.integers(-20, 20))
        b = f32(rng.standard_normal() * 10.0 ** rng.integers(-20, 20))
        if rng.random() < 0.3:
            b = f32(-a * (1 + 2.0 ** -rng.integers(1, 24)))  # heavy cancellation
        pairs.append((a, b))
    res = run(driver, [f"ts {a.hex()} {b.hex()}" for a, b in pairs])
    for (a, b), (s, e) in zip(pairs, res):
        assert Fraction(s) + Fraction(e) == Fraction(a) + Fraction(b)
        assert s == f32(a + b)  # s is the rounded sum


def _split(x):
    hi = f32(x)
    return hi, f32(x - hi)


@pytest.mark.parametrize("op", ["add", "mul"])
def test_double_float_add_and_mul(driver, op):
    rng = np.random.default_rng(2 if op == "add" else 3)
    cases = []
    for _ in range(2000):
        x = rng.standard_normal() * 10.0 ** rng.integers(-8, 8)
        y = rng.standard_normal() * 10.0 ** rng.integers(-8, 8)
        if op == "add" and rng.random() < 0.3:
            y = -x * (1 + 1e-6 * rng.standard_normal())
        cases.append((_split(x), _split(y)))
    res = run(driver, [f"{op} {a[0].hex()} {a[1].hex()} {b[0].hex()} {b[1].hex()}" for a, b in cases])
    for (a, b), (hi, lo) in zip(cases, res):
        fa, fb = Fraction(a[0]) + Fraction(a[1]), Fraction(b[0]) + Fraction(b[1])
        exact = fa + fb if op == "add" else fa * fb
        got = Fraction(hi) + Fraction(lo)
        scale = abs(fa) + abs(fb) if op == "add" else abs(fa * fb)
        assert abs(got - exact) <= Fraction(2) ** -44 * scale, (op, a, b)
        assert abs(lo) <= abs(hi) * 2.0 ** -23 + 1e-300  # normalised


def test_double_float_accumulation(driver):
    rng = np.random.default_rng(4)
    lines, sums = [], []
    for n in (10, 1000, 20000):
        xs = rng.standard_normal(n) * np.exp(rng.uniform(-5, 5, n))
        lines.append(f"acc {n} " + " ".join(float(x).hex() for x in xs))
        sums.append((sum(Fraction(_split(x)[0]) + Fraction(_split(x)[1]) for x in xs), float(np.sum(np.abs(xs)))))
    for (exact, mag), (hi, lo) in zip(sums, run(driver, lines)):
        assert abs(float(Fraction(hi) + Fraction(lo) - exact)) <= 1e-12 * mag


def _rotation(rng):
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    return q


def test_spd_block_inverse(driver):
    rng = np.random.default_rng(5)
    mats, kinds = [], []
    for t in range(400):
        q = _rotation(rng)
        kind = t % 4
        lam = np.array([1.0, 0.5 + abs(rng.standard_normal()), 0.3 + abs(rng.standard_normal())])
        if kind == 1:
            lam[1:] = [1e-6, 3e-7]     # nearly singular, SPD
        elif kind == 2:
            lam[1] = -2e-6             # slightly indefinite (rounding of a Galerkin sum)
        elif kind == 3:
            lam[:] = 0.0               # no stiffness at all
        a = (q * lam) @ q.T
        mats.append(a.astype(np.float32).astype(np.float64))  # the kernel sees FP32 stencils
        kinds.append(kind)
    res = run(driver, ["inv " + " ".join(float(v).hex() for v in m.ravel()) for m in mats])
    for a, kind, o in zip(mats, kinds, res):
        o = np.array(o).reshape(3, 3)
        if kind == 3:
            assert not o.any()
            continue
        assert np.allclose(o, o.T, rtol=0, atol=1e-12 * np.abs(o).max())
        ev = np.linalg.eigvalsh(o.astype(np.float32).astype(np.float64))  # SPD after FP32 storage
        assert ev.min() > 0.0
        lmax = np.abs(np.linalg.eigvalsh(0.5 * (a + a.T))).max()
        assert ev.max() <= 1.01 / (1e-5 * lmax)  # eigenvalues floored at 1e-5 |lambda|_max
        if kind == 0:
            assert np.abs(o @ a - np.eye(3)).max() <= 1e-9
