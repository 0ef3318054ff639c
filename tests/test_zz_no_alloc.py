"""The entry point that allocates no memory, for callers that cannot allocate device
memory while they step the model (a solver run inside another framework's callback,
or a service that forbids allocation after start-up): it must give the same state as
the regular hierarchy entry points, call after call, with its working memory in a
static device array shared by all calls.

This file is collected last so that a stop at the first failure has already run every
other test; it passes alone in a fresh process too.
"""
import ctypes

import numpy as np
import pytest

from paper_1803_01450_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-11


def _rel(a, b):
    den = np.maximum(np.abs(b).max(axis=(1, 2)), 1e-300)
    return (np.abs(a - b).max(axis=(1, 2)) / den).max()


def test_noalloc_step_matches_hierarchy_two_calls(mlswe_lib):
    import torch

    pkg = mlswe_lib
    L = pkg.lib()
    fn = L.mlswe_step_fixed_noalloc
    fn.argtypes = [ctypes.POINTER(pkg._Config), ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                   ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.POINTER(ctypes.c_double)]
    fn.restype = ctypes.c_int

    ny, nx = 96, 160
    q0, B = I.gaussian_random_state(21, 2, nx, ny)
    dx, dy = 1.0 / nx, 1.0 / ny
    dt = 0.2 * min(dx, dy) / 4.0
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

    # Sizes beyond the static array are rejected with EINVAL before any GPU work.
    st = fn(ctypes.byref(ccfg), 1024, 1024, dx, dy, dt, a.data_ptr(), Bt.data_ptr(), b.data_ptr(), stream, None)
    assert st == 1
