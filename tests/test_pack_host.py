"""The packed sweep tiles of the batched form (host code, compiled here without a GPU): the
runs of a patch cover its lines and their ghost lines exactly once with the right flags,
and the packing keeps every run's lines in order, respects the sweep kernel's shared-memory
limits (256 edges, 288 cells, 4 groups of one (member, level) per tile) and closes a tile
only when the next line cannot join it."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
MAX_EDGES, MAX_CELLS, MAX_GROUPS = 256, 288, 4


@pytest.fixture(scope="module")
def pk(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not found")
    so = str(tmp_path_factory.mktemp("pk") / "libpk.so")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-shared", "-Xcompiler", "-fPIC", "-o", so,
                    os.path.join(HERE, "pack_host_check.cu"),
                    os.path.join(ROOT, "paper_1803_01450_gb300", "csrc", "mlswe_pack.cu")],
                   check=True, capture_output=True)
    L = ctypes.CDLL(so)
    ip = ctypes.POINTER(ctypes.c_int)
    L.pk_segments.argtypes = [ctypes.c_int] * 9 + [ip, ctypes.c_int]
    L.pk_segments.restype = ctypes.c_int
    L.pk_pack.argtypes = [ip, ctypes.c_int, ctypes.c_int, ip, ctypes.c_int, ip, ctypes.c_int, ip]
    L.pk_pack.restype = ctypes.c_int
    return L


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def segments(pk, box, dir_, tile_len, g0, g1, desc):
    out = np.zeros(6 * 4096, np.int32)
    n = pk.pk_segments(*box, dir_, tile_len, g0, g1, desc, _ip(out), 4096)
    assert n <= 4096
    return out[:6 * n].reshape(n, 6)


def pack(pk, segs, dir_):
    segs = np.ascontiguousarray(segs, np.int32)
    n_lines = int(segs[:, 4].sum()) if len(segs) else 0
    items = np.zeros(6 * max(1, n_lines), np.int32)
    toff = np.zeros(n_lines + 2, np.int32)
    counts = np.zeros(2, np.int32)
    rc = pk.pk_pack(_ip(segs), len(segs), dir_, _ip(items), n_lines, _ip(toff), n_lines + 2, _ip(counts))
    if rc == 0:
        return None
    assert rc == 1
    return items[:6 * counts[0]].reshape(-1, 6), toff[:counts[1] + 1]


def line_parts(rows, dir_):
    """(desc, line, start along, len, flags) of every line of every run or group, in order."""
    out = []
    for desc, i0, j0, ln, nl, fl in rows:
        for k in range(nl):
            line, a = (j0 + k, i0) if dir_ == 0 else (i0 + k, j0)
            out.append((desc, line, a, ln, fl))
    return out


def random_layout(rng, n, side, count):
    boxes, taken = [], np.zeros((n, n), bool)
    for _ in range(count * 20):
        if len(boxes) == count:
            break
        w, h = (int(x) for x in rng.integers(side[0], side[1] + 1, 2))
        if w > n or h > n:
            continue
        i0, j0 = int(rng.integers(0, n - w + 1)), int(rng.integers(0, n - h + 1))
        if taken[j0:j0 + h, i0:i0 + w].any():
            continue
        taken[j0:j0 + h, i0:i0 + w] = True
        boxes.append((i0, j0, i0 + w, j0 + h))
    return boxes


def ghost_lines(box, dir_, mode, n):
    lo, hi = (box[1], box[3]) if dir_ == 0 else (box[0], box[2])
    if mode == "unsplit":
        return lo - 1, hi + 1
    if mode == "refined" and dir_ == 0:
        return max(0, lo - 2), min(n, hi + 2)
    return lo, hi


@pytest.mark.parametrize("dir_", [0, 1])
@pytest.mark.parametrize("mode", ["plain", "refined", "unsplit"])
def test_runs_cover_each_line_once(pk, dir_, mode):
    rng = np.random.default_rng(7 + dir_ + 10 * len(mode))
    n = 160
    for box in random_layout(rng, n, (16, 64), 12):
        tile_len = int(rng.choice([253, 125, 61, 29, int(rng.integers(4, 70))]))
        g0, g1 = ghost_lines(box, dir_, mode, n)
        segs = segments(pk, box, dir_, tile_len, g0, g1, desc=3)
        a0, a1 = (box[0], box[2]) if dir_ == 0 else (box[1], box[3])
        lo, hi = (box[1], box[3]) if dir_ == 0 else (box[0], box[2])
        seen = np.zeros((g1 - g0, a1 - a0), np.int32)
        for desc, line, a, ln, fl in line_parts(segs, dir_):
            assert desc == 3 and 1 <= ln <= tile_len
            seen[line - g0, a - a0:a - a0 + ln] += 1
            assert (fl & 1) == (1 if lo <= line < hi else 0)
            assert (fl >> 1 & 1) == (1 if a + ln == a1 else 0)
        assert (seen == 1).all()


@pytest.mark.parametrize("seed", range(8))
def test_packing_limits_order_and_greed(pk, seed):
    rng = np.random.default_rng(100 + seed)
    dir_ = seed % 2
    mode = ["plain", "refined", "unsplit"][seed % 3]
    n = 200
    segs = []
    for desc in range(int(rng.integers(1, 4))):  # members / levels: one desc each
        tile_len = int(rng.choice([253, 125, 61, 29, int(rng.integers(4, 120))]))
        for box in random_layout(rng, n, (16, 64), int(rng.integers(1, 25))):
            g0, g1 = ghost_lines(box, dir_, mode, n)
            segs.append(segments(pk, box, dir_, tile_len, g0, g1, desc))
    segs = np.concatenate(segs)
    items, toff = pack(pk, segs, dir_)
    # every line of every run, once, in the runs' order, with its flags
    assert line_parts(items, dir_) == line_parts(segs, dir_)
    assert toff[0] == 0 and toff[-1] == len(items) and (np.diff(toff) >= 1).all()
    for t in range(len(toff) - 1):
        g = items[toff[t]:toff[t + 1]]
        assert 1 <= len(g) <= MAX_GROUPS
        assert (g[:, 0] == g[0, 0]).all()
        edges = int((g[:, 4] * (g[:, 3] + 3)).sum())
        cells = int((g[:, 4] * (g[:, 3] + 4)).sum())
        assert edges <= MAX_EDGES and cells <= MAX_CELLS
        if t + 2 < len(toff):  # greedy: the next group's first line did not fit this tile
            nx = items[toff[t + 1]]
            fits = (edges + nx[3] + 3 <= MAX_EDGES and cells + nx[3] + 4 <= MAX_CELLS
                    and len(g) < MAX_GROUPS and nx[0] == g[0, 0])
            assert not fits
    # no tile count below the edge bound
    total_edges = int((segs[:, 4] * (segs[:, 3] + 3)).sum())
    assert len(toff) - 1 >= -(-total_edges // MAX_EDGES)


def test_single_large_patch_tile_count(pk):
    """A 2048^2 patch swept along x with 253-cell parts: 8 full parts of one line per tile and
    a 24-cell part of nine lines per tile (9 x 27 = 243 edges)."""
    segs = segments(pk, (0, 0, 2048, 2048), 0, 253, 0, 2048, 0)
    items, toff = pack(pk, segs, 0)
    assert len(toff) - 1 == 8 * 2048 + -(-2048 // 9)


def test_line_longer_than_a_tile_is_refused(pk):
    segs = np.array([[0, 0, 0, 254, 3, 1]], np.int32)
    assert pack(pk, segs, 0) is None
    segs = np.array([[0, 0, 0, 253, 3, 1]], np.int32)
    items, toff = pack(pk, segs, 0)
    assert len(toff) - 1 == 3


def test_empty_input(pk):
    items, toff = pack(pk, np.zeros((0, 6), np.int32), 0)
    assert len(items) == 0 and list(toff) == [0]
