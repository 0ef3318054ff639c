"""The sweep kernel's reciprocal, reciprocal square root and square root by iteration (FP32
seed and one third-order Newton-Raphson step where |x| lies in [2^-160, 2^160), the library
functions elsewhere) against an exact reference (50-digit decimal arithmetic, correctly
rounded back to FP64) and against CUDA's own functions: at most one unit in the last place
from the correctly rounded value, and the library's values where the iteration does not run
(zero, subnormals, huge and non-finite arguments, negative square roots). And the share of a
limited wave that goes to the left cell, whose weight carries the MC limiter's factor 2,
against the second-order correction written out as in the wave-propagation method:
base + sign(s) (1 - nu |s|) phi(theta) / 2."""
import ctypes
import decimal
import os
import shutil
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def mc(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    so = str(tmp_path_factory.mktemp("mc") / "libmc.so")
    subprocess.run([nvcc, "-std=c++17", "-O3", "-shared", "-Xcompiler", "-fPIC",
                    "-gencode", "arch=compute_103a,code=sm_103a", "-o", so, os.path.join(HERE, "math_check.cu")],
                   check=True, capture_output=True)
    L = ctypes.CDLL(so)
    dp = ctypes.POINTER(ctypes.c_double)
    L.mc_run.argtypes = [dp, ctypes.c_int, dp]
    L.mc_run.restype = ctypes.c_int
    L.mc_left_share.argtypes = [dp, ctypes.POINTER(ctypes.c_int), ctypes.c_int, dp]
    L.mc_left_share.restype = ctypes.c_int
    L.mc_solve.argtypes = [dp, ctypes.c_int, dp]
    L.mc_solve.restype = ctypes.c_int
    return L


def run(mc, x):
    x = np.ascontiguousarray(x, np.float64)
    out = np.zeros((6, len(x)))
    dp = ctypes.POINTER(ctypes.c_double)
    assert mc.mc_run(x.ctypes.data_as(dp), len(x), out.ctypes.data_as(dp)) == 0
    return out


def ulps(a, b):
    """Distance in units in the last place between doubles of the same sign."""
    ia, ib = a.view(np.int64), b.view(np.int64)
    return np.abs(ia - ib)


def exact(x, kind):
    decimal.getcontext().prec = 50
    out = np.empty_like(x)
    for k, v in enumerate(x):
        d = decimal.Decimal(float(v))
        if kind == "rcp":
            r = 1 / d
        elif kind == "rsqrt":
            r = 1 / d.sqrt()
        else:
            r = d.sqrt()
        out[k] = float(r)  # correctly rounded
    return out


def moderate_inputs(rng, n, positive):
    e = rng.uniform(-159.5, 159.5, n)
    x = np.exp2(e) * rng.uniform(1.0, 2.0, n)
    x = np.concatenate([x, 1.0 + np.arange(64) * 2.0 ** -20, [1.0, 2.0, 4.0, 0.5, 3.0, 1.5, 2.0 ** 159, 2.0 ** -160]])
    if not positive:
        x = x * np.where(rng.random(len(x)) < 0.5, -1.0, 1.0)
    return x


def test_reciprocal_within_one_ulp(mc):
    rng = np.random.default_rng(11)
    x = moderate_inputs(rng, 200000, positive=False)
    out = run(mc, x)
    assert (ulps(out[0], out[1]) <= 1).all()  # CUDA's __drcp_rn is correctly rounded
    s = x[:3000]
    assert (ulps(out[0][:3000], exact(s, "rcp")) <= 1).all()


def test_reciprocal_square_root_and_square_root_within_one_ulp(mc):
    rng = np.random.default_rng(12)
    x = moderate_inputs(rng, 200000, positive=True)
    out = run(mc, x)
    s = x[:3000]
    assert (ulps(out[2][:3000], exact(s, "rsqrt")) <= 1).all()
    assert (ulps(out[4][:3000], exact(s, "sqrt")) <= 2).all()  # x times an rsqrt within one ulp
    # against CUDA's rsqrt (itself within one ulp) and correctly rounded sqrt, on all inputs
    assert (ulps(out[2], out[3]) <= 2).all()
    assert (ulps(out[4], out[5]) <= 2).all()


def test_outside_the_range_the_library_functions_answer(mc):
    tiny = np.nextafter(0.0, 1.0)
    x = np.array([0.0, -0.0, tiny, 1e-300, 2.0 ** -161, 2.0 ** 161, 1e300, np.inf, -np.inf, np.nan, -1.0, -4.0,
                  -2.0 ** -170, 2.0 ** -170])
    out = run(mc, x)
    for fast, ref in ((0, 1), (2, 3), (4, 5)):
        a, b = out[fast], out[ref]
        for k, v in enumerate(x):
            if fast == 0 and 2.0 ** -160 <= abs(v) < 2.0 ** 161:
                continue  # -1, -4 are in range for the reciprocal
            assert (np.isnan(a[k]) and np.isnan(b[k])) or a[k].view(np.int64) == b[k].view(np.int64), (fast, v)
    inr = np.abs(x) >= 2.0 ** -160
    inr &= np.abs(x) < 2.0 ** 161
    assert (ulps(out[0][inr], out[1][inr]) <= 1).all()


def _phi(kind, th):
    if kind == 0:
        return 1.0
    if th <= 0.0:
        return 0.0
    if kind == 1:
        return min(1.0, th)
    return max(0.0, min(0.5 * (1.0 + th), 2.0, 2.0 * th))


def test_left_share_matches_the_written_out_correction(mc):
    rng = np.random.default_rng(13)
    n = 60000
    kind = rng.integers(0, 3, n)
    sc = rng.choice([-1, 0, 1], n, p=[0.45, 0.1, 0.45])
    act = (rng.random(n) < 0.9) & (sc != 0)
    s = sc * np.exp2(rng.uniform(-8, 4, n))
    nu = rng.uniform(0.0, 0.9, n) / np.maximum(np.abs(s), 1e-300)
    nu = np.where(sc == 0, rng.uniform(0.0, 1.0, n), nu)
    # theta spanning the limiter's kinks (0, 1/3, 1, 3) and both signs
    th = np.concatenate([rng.uniform(-2, 6, n // 2), rng.choice([0.0, 1 / 3, 1.0, 3.0, -0.0], n - n // 2)])
    th = th * (1.0 + rng.uniform(-1e-12, 1e-12, n))
    num = th * np.exp2(rng.integers(-20, 20, n))
    iden = np.where(th == 0, 1.0, th / np.where(num == 0, 1.0, num))
    inp = np.ascontiguousarray(np.stack([num, iden, s, nu], axis=1))
    fl = np.ascontiguousarray(np.stack([kind, sc, act.astype(int)], axis=1).astype(np.int32))
    out = np.zeros(n)
    dp = ctypes.POINTER(ctypes.c_double)
    assert mc.mc_left_share(inp.ctypes.data_as(dp), fl.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), n,
                            out.ctypes.data_as(dp)) == 0
    for k in range(n):
        base = 1.0 if sc[k] < 0 else (0.0 if sc[k] > 0 else 0.5)
        ref = base
        if act[k]:
            t = num[k] * iden[k]  # theta as the kernel forms it
            ref = base + (0.5 if sc[k] > 0 else -0.5) * (1.0 - nu[k] * abs(s[k])) * _phi(kind[k], t)
        # a few roundings apart (the kernel fuses; the written-out form rounds each step)
        assert abs(out[k] - ref) <= 1e-15 * max(1.0, abs(ref)), (k, kind[k], sc[k], act[k], out[k], ref)


def test_elimination_for_two_right_hand_sides_equals_two_solves(mc):
    """The transverse solve of three layers eliminates the eigenvector matrix once for both
    fluctuations: the same pivots and operations per right-hand side as two separate solves,
    so the same bits; and the solution solves the system (against numpy)."""
    rng = np.random.default_rng(14)
    n = 4000
    A = rng.standard_normal((n, 6, 6))
    A[: n // 4] *= np.exp2(rng.integers(-20, 20, (n // 4, 6, 1)))  # badly scaled rows: pivoting
    A[n // 4: n // 2, :, 0] *= 1e-9  # small leading column: row exchanges
    b = rng.standard_normal((n, 2, 6))
    inp = np.ascontiguousarray(np.concatenate([A.reshape(n, 36), b.reshape(n, 12)], axis=1))
    out = np.zeros((n, 24))
    dp = ctypes.POINTER(ctypes.c_double)
    assert mc.mc_solve(inp.ctypes.data_as(dp), n, out.ctypes.data_as(dp)) == 0
    single, multi = out[:, :12], out[:, 12:]
    assert np.array_equal(single.view(np.int64), multi.view(np.int64))
    x = np.linalg.solve(A, b.transpose(0, 2, 1)).transpose(0, 2, 1).reshape(n, 12)
    cond = np.linalg.cond(A)
    ok = cond < 1e8
    err = np.abs(single - x).max(axis=1) / np.maximum(np.abs(x).max(axis=1), 1e-300)
    assert (err[ok] <= 1e-15 * cond[ok] * 100).all()
