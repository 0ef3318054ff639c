"""The entry point that allocates no memory, for callers that cannot allocate device
memory while they step the model (a solver run inside another framework's callback,
or a service that forbids allocation after start-up): it must give the same state as
the regular hierarchy entry points and as the oracle, call after call, with its working
memory in a static device array shared by all calls, and it must allocate nothing.

This file is collected last so that a stop at the first failure has already run every
other test; it passes alone in a fresh process too.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_1803_01450_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-11
EINVAL = 1


def _rel(a, b):
    den = np.maximum(np.abs(b).max(axis=(1, 2)), 1e-300)
    return (np.abs(a - b).max(axis=(1, 2)) / den).max()


def _entry(pkg):
    fn = pkg.lib().mlswe_step_fixed_noalloc
    fn.argtypes = [ctypes.POINTER(pkg._Config), ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                   ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.POINTER(ctypes.c_double)]
    fn.restype = ctypes.c_int
    return fn


def _case():
    ny, nx = 96, 160
    q0, B = I.gaussian_random_state(21, 2, nx, ny)
    dx, dy = 1.0 / nx, 1.0 / ny
    dt = 0.2 * min(dx, dy) / 4.0
    return nx, ny, q0, B, dx, dy, dt


def test_noalloc_step_matches_hierarchy_two_calls(mlswe_lib):
    import torch

    pkg = mlswe_lib
    fn = _entry(pkg)
    nx, ny, q0, B, dx, dy, dt = _case()
    cfg = pkg.Config(M=2, dry_tol=1e-6, order=2, limiter=2, max_levels=1)

    # Regular path: hierarchy (allocates its own working memory), two steps.
    H = pkg.Hierarchy(cfg, [(0.0, 0.0, nx * dx, ny * dy, nx, ny)])
    H.set_bathymetry(0, B)
    H.set_state(0, 0, q0)
    H.step_level(0, dt=dt)
    ref1 = H.get_state(0, 0)
    H.step_level(0, dt=dt)
    ref2 = H.get_state(0, 0)
    H.close()

    # No-allocation path: caller-owned device buffers, two calls in a row.
    dev = torch.device("cuda", 0)
    a = torch.tensor(q0, dtype=torch.float64, device=dev).contiguous()
    b = torch.empty_like(a)
    c = torch.empty_like(a)
    Bt = torch.tensor(B, dtype=torch.float64, device=dev).contiguous()
    stream = torch.cuda.current_stream(dev).cuda_stream
    ccfg = cfg.to_c()
    cfl = ctypes.c_double(0.0)
    st = fn(ctypes.byref(ccfg), nx, ny, dx, dy, dt, a.data_ptr(), Bt.data_ptr(), b.data_ptr(), stream, ctypes.byref(cfl))
    assert st == 0, st
    st = fn(ctypes.byref(ccfg), nx, ny, dx, dy, dt, b.data_ptr(), Bt.data_ptr(), c.data_ptr(), stream, None)
    assert st == 0, st
    torch.cuda.synchronize()
    out1 = b.cpu().numpy()
    out2 = c.cpu().numpy()
    assert _rel(out1, ref1) <= TOL
    assert _rel(out2, ref2) <= TOL
    assert 0.0 < cfl.value < 1.0

    # And against the oracle directly (the FP64 CPU implementation), step by step.
    P = O.params(M=2, dry_tol=1e-6, order=2, limiter=2)
    o1, _, _ = O.step_walled(P, q0, B, dx, dy, dt)
    o2, _, _ = O.step_walled(P, o1, B, dx, dy, dt)
    assert _rel(out1, o1) <= TOL
    assert _rel(out2, o2) <= TOL

    # Sizes beyond the static array are rejected with EINVAL before any GPU work.
    st = fn(ctypes.byref(ccfg), 1024, 1024, dx, dy, dt, a.data_ptr(), Bt.data_ptr(), b.data_ptr(), stream, None)
    assert st == EINVAL


RHO = {1: (1000.0,), 3: (1000.0, 1020.0, 1030.0), 4: (1000.0, 1020.0, 1030.0, 1040.0)}


@pytest.mark.parametrize("M", [1, 3, 4])
def test_noalloc_step_matches_oracle_other_layer_counts(mlswe_lib, M):
    """One, three and four layers (Eqs. (4)-(5) for any M): three calls in a row against the
    oracle's walled step, each field within 1e-11 of its scale; the size limit is by layer
    cells (M nx ny <= 2 x 512 x 512)."""
    import torch
    from conftest import report, state_err

    pkg = mlswe_lib
    fn = _entry(pkg)
    ny, nx = 57, 90
    depth = {1: (0.5,), 3: (0.4, 0.3, 0.6), 4: (0.4, 0.3, 0.35, 0.6)}[M]
    q0, B = I.gaussian_random_state(60 + M, M, nx, ny, depth=depth, vel=0.01)
    dx, dy = 1.0 / nx, 1.2 / ny
    dt = 0.2 * min(dx, dy) / 4.0
    ccfg = pkg.Config(M=M, rho=RHO[M], dry_tol=1e-6, order=2, limiter=2, max_levels=1).to_c()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev).cuda_stream
    a = torch.tensor(q0, dtype=torch.float64, device=dev).contiguous()
    b = torch.empty_like(a)
    Bt = torch.tensor(B, dtype=torch.float64, device=dev).contiguous()
    P = O.params(M=M, rho=RHO[M], dry_tol=1e-6, order=2, limiter=2)
    qo = q0.copy()
    for k in range(3):
        src, dst = (a, b) if k % 2 == 0 else (b, a)
        assert fn(ctypes.byref(ccfg), nx, ny, dx, dy, dt, src.data_ptr(), Bt.data_ptr(), dst.data_ptr(), stream,
                  None) == 0
        qo, _, _ = O.step_walled(P, qo, B, dx, dy, dt)
    torch.cuda.synchronize()
    err = state_err(b.cpu().numpy(), qo, M)
    report(f"noalloc_M{M}_{ny}x{nx}_3steps", err)
    assert err.max() < TOL, err
    side = int((2 * 512 * 512 // M) ** 0.5)
    rows = 2 * 512 * 512 // (M * side) + 1  # one row more than the array holds
    assert M * side * (rows - 1) <= 2 * 512 * 512 < M * side * rows
    assert fn(ctypes.byref(ccfg), side, rows, dx, dy, dt, a.data_ptr(), Bt.data_ptr(), b.data_ptr(), stream,
              None) == EINVAL


def test_noalloc_rejects_host_and_overlapping_buffers(mlswe_lib):
    """Host arrays (which a kernel would fault on) and an output that overlaps an input are
    refused with EINVAL before any launch; the outputs stay untouched."""
    import torch

    pkg = mlswe_lib
    fn = _entry(pkg)
    nx, ny, q0, B, dx, dy, dt = _case()
    ccfg = pkg.Config(M=2, dry_tol=1e-6, order=2, limiter=2, max_levels=1).to_c()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev).cuda_stream
    a = torch.tensor(q0, dtype=torch.float64, device=dev).contiguous()
    Bt = torch.tensor(B, dtype=torch.float64, device=dev).contiguous()
    out = torch.full_like(a, 7.0)
    qh = np.ascontiguousarray(q0)
    Bh = np.ascontiguousarray(B)
    oh = np.full_like(qh, 7.0)
    host_cases = [(qh.ctypes.data, Bt.data_ptr(), out.data_ptr()),
                  (a.data_ptr(), Bh.ctypes.data, out.data_ptr()),
                  (a.data_ptr(), Bt.data_ptr(), oh.ctypes.data)]
    for q_in, b_in, q_out in host_cases:
        assert fn(ctypes.byref(ccfg), nx, ny, dx, dy, dt, q_in, b_in, q_out, stream, None) == EINVAL
    # overlaps: the output starting inside the input state, the same buffer, inside B
    big = torch.zeros(2 * a.numel(), dtype=torch.float64, device=dev)
    big[:a.numel()] = a.reshape(-1)
    half = big.data_ptr() + 8 * (a.numel() // 2)
    Bbig = torch.zeros(a.numel(), dtype=torch.float64, device=dev)
    for q_in, b_in, q_out in [(big.data_ptr(), Bt.data_ptr(), half),
                              (a.data_ptr(), Bt.data_ptr(), a.data_ptr()),
                              (a.data_ptr(), Bbig.data_ptr(), Bbig.data_ptr() + 8 * 5)]:
        assert fn(ctypes.byref(ccfg), nx, ny, dx, dy, dt, q_in, b_in, q_out, stream, None) == EINVAL
    torch.cuda.synchronize()
    assert bool((out == 7.0).all()) and np.all(oh == 7.0)


def test_noalloc_allocates_nothing(mlswe_lib):
    """After a first call (which looks up the static array's address), further calls, with
    and without the Courant report, leave the device's free memory unchanged."""
    import torch

    pkg = mlswe_lib
    fn = _entry(pkg)
    nx, ny, q0, B, dx, dy, dt = _case()
    ccfg = pkg.Config(M=2, dry_tol=1e-6, order=2, limiter=2, max_levels=1).to_c()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev).cuda_stream
    a = torch.tensor(q0, dtype=torch.float64, device=dev).contiguous()
    b = torch.empty_like(a)
    Bt = torch.tensor(B, dtype=torch.float64, device=dev).contiguous()
    cfl = ctypes.c_double(0.0)
    assert fn(ctypes.byref(ccfg), nx, ny, dx, dy, dt, a.data_ptr(), Bt.data_ptr(), b.data_ptr(), stream, None) == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    for k in range(6):
        src, dst = (a, b) if k % 2 == 0 else (b, a)
        out_cfl = ctypes.byref(cfl) if k % 3 == 0 else None
        assert fn(ctypes.byref(ccfg), nx, ny, dx, dy, dt, src.data_ptr(), Bt.data_ptr(), dst.data_ptr(), stream,
                  out_cfl) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(dev)[0] == free0
