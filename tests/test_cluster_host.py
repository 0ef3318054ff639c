"""The library's flag dilation and Berger-Rigoutsos clustering (host code, compiled here
without a GPU) against the oracle's: identical flags after dilation and identical boxes on
random flag fields of several sizes, densities and shapes (blobs and scattered cells), on a
level 0 domain and inside the nesting regions of a refined level."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import cluster as C

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def hc(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not found")
    so = str(tmp_path_factory.mktemp("hc") / "libhc.so")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-shared", "-Xcompiler", "-fPIC", "-o", so,
                    os.path.join(HERE, "cluster_host_check.cu"),
                    os.path.join(ROOT, "paper_1803_01450_gb300", "csrc", "mlswe_cluster.cu")],
                   check=True, capture_output=True)
    L = ctypes.CDLL(so)
    u8 = ctypes.POINTER(ctypes.c_uint8)
    ip = ctypes.POINTER(ctypes.c_int)
    L.hc_dilate.argtypes = [u8, ctypes.c_int, ctypes.c_int, ctypes.c_int, u8]
    L.hc_cluster.argtypes = [u8, ctypes.c_int, ctypes.c_int, ctypes.c_int, ip, ctypes.c_int, ctypes.c_int,
                             ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, ip, ctypes.c_int]
    L.hc_cluster.restype = ctypes.c_int
    L.hc_fresh.argtypes = [ip, ctypes.c_int, ip, ctypes.c_int, ip, ctypes.c_int]
    L.hc_fresh.restype = ctypes.c_int
    return L


def _u8(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _flags(rng, ny, nx, kind):
    if kind == "scatter":
        return (rng.random((ny, nx)) < rng.uniform(0.001, 0.05)).astype(np.uint8)
    f = np.zeros((ny, nx), np.uint8)
    y, x = np.mgrid[0:ny, 0:nx]
    for _ in range(int(rng.integers(1, 6))):
        cx, cy, rad = rng.uniform(0, nx), rng.uniform(0, ny), rng.uniform(2, 0.3 * min(nx, ny))
        ring = kind == "rings"
        d = np.hypot(x - cx, y - cy)
        f |= ((np.abs(d - rad) < 1.5) if ring else (d < rad)).astype(np.uint8)
    return f


@pytest.mark.parametrize("seed", range(12))
def test_dilation_matches_oracle(hc, seed):
    rng = np.random.default_rng(seed)
    ny, nx = int(rng.integers(1, 90)), int(rng.integers(1, 90))
    f = _flags(rng, ny, nx, ["scatter", "blobs", "rings"][seed % 3])
    for n in (0, 1, 2, 3):
        out = np.zeros_like(f)
        hc.hc_dilate(_u8(f), nx, ny, n, _u8(out))
        assert np.array_equal(out.astype(bool), C.dilate(f, n)), (seed, n)


@pytest.mark.parametrize("seed", range(16))
def test_clustering_matches_oracle(hc, seed):
    rng = np.random.default_rng(100 + seed)
    r = [2, 4][seed % 2]
    level = 0 if seed < 8 else 1
    nx, ny = int(rng.integers(24, 160)), int(rng.integers(24, 160))
    f = _flags(rng, ny, nx, ["scatter", "blobs", "rings"][seed % 3])
    if level == 0:
        patches = [(0, 0, nx, ny)]
    else:  # a few disjoint patches of the flagged level
        patches = []
        for _ in range(int(rng.integers(1, 5))):
            i0, j0 = int(rng.integers(0, nx - 12)), int(rng.integers(0, ny - 12))
            b = (i0, j0, min(nx, i0 + int(rng.integers(12, 60))), min(ny, j0 + int(rng.integers(12, 60))))
            if all(b[2] <= p[0] or p[2] <= b[0] or b[3] <= p[1] or p[3] <= b[1] for p in patches):
                patches.append(b)
    min_side, max_side = 4 * r, 16 * r
    want = C.cluster(f, level, patches, r, 2, 0.7, min_side, max_side, 2)
    pa = np.ascontiguousarray(np.array(patches, dtype=np.int32).reshape(-1, 4))
    cap = 4 * nx * ny
    out = np.zeros((cap, 4), np.int32)
    n = hc.hc_cluster(_u8(f), nx, ny, level, pa.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), len(patches), r, 2,
                      0.7, min_side, max_side, 2, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), cap)
    assert [tuple(b) for b in out[:n].tolist()] == [tuple(b) for b in want]


def _disjoint_boxes(rng, n, nx, ny, lo, hi):
    occ = np.zeros((ny, nx), bool)
    out = []
    for _ in range(20 * n):
        if len(out) == n:
            break
        w, h = (int(v) for v in rng.integers(lo, hi + 1, 2))
        i0, j0 = int(rng.integers(0, nx - w + 1)), int(rng.integers(0, ny - h + 1))
        if not occ[j0:j0 + h, i0:i0 + w].any():
            occ[j0:j0 + h, i0:i0 + w] = True
            out.append((i0, j0, i0 + w, j0 + h))
    return out


@pytest.mark.parametrize("seed", range(6))
def test_fresh_cells_are_new_minus_old(hc, seed):
    """The regrid fills the cells of the new layout that no old patch held: the boxes the
    library returns are disjoint and cover exactly those cells (boxes spanning several
    64-cell buckets and none at all included)."""
    rng = np.random.default_rng(700 + seed)
    nx, ny = 300, 260
    new = _disjoint_boxes(rng, int(rng.integers(0, 60)), nx, ny, 4, 90)
    old = _disjoint_boxes(rng, int(rng.integers(0, 60)), nx, ny, 4, 90)
    ip = ctypes.POINTER(ctypes.c_int)
    a = np.ascontiguousarray(np.array(new, dtype=np.int32).reshape(-1, 4))
    b = np.ascontiguousarray(np.array(old, dtype=np.int32).reshape(-1, 4))
    cap = 100000
    out = np.zeros((cap, 4), np.int32)
    n = hc.hc_fresh(a.ctypes.data_as(ip), len(new), b.ctypes.data_as(ip), len(old), out.ctypes.data_as(ip), cap)
    cnt = np.zeros((ny, nx), np.int32)
    for (i0, j0, i1, j1) in out[:n].tolist():
        assert i0 < i1 and j0 < j1
        cnt[j0:j1, i0:i1] += 1
    want = np.zeros((ny, nx), bool)
    for (i0, j0, i1, j1) in new:
        want[j0:j1, i0:i1] = True
    for (i0, j0, i1, j1) in old:
        want[j0:j1, i0:i1] = False
    assert cnt.max() <= 1 and np.array_equal(cnt.astype(bool), want)
