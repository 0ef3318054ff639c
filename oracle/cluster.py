"""Deterministic Berger-Rigoutsos clustering of refinement flags (oracle side).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper defers flagging and clustering to GeoClaw's AMR (Sec. 2: "the
management of these finer and coarser meshes is adaptive"; the algorithm is
in its reference [an]). This module is this project's deterministic reading,
written so that two independent implementations give the same boxes:

* flags are dilated by ``n_buf`` cells (Chebyshev distance), then restricted
  to the region where a finer patch may be placed: for level 0 the domain, for
  a refined level each of its patches shrunk by ``n_nest`` cells on the sides
  that do not touch the domain boundary; every region is clustered on its own;
* in a box: take the bounding box of its flags, grow it to ``min_len`` per side
  inside the box (upper side first); accept it when its efficiency (flags /
  area) is at least ``eff`` and both sides are at most ``max_len``;
* otherwise split it: at the first hole of a signature (the longer side's
  dimension first, x on ties), else at the strongest sign change of the
  signature's second difference (ties: dimension order, then lowest position),
  else at the middle of the longer side; a split never leaves a part shorter
  than ``min_len``; if none is possible the box is accepted as is;
* boxes are returned sorted by (j0, i0). Boxes are half-open (i0, j0, i1, j1).
"""
from __future__ import annotations

import numpy as np


def dilate(flags: np.ndarray, n: int) -> np.ndarray:
    ny, nx = flags.shape
    out = np.zeros_like(flags, dtype=bool)
    f = flags.astype(bool)
    for dj in range(-n, n + 1):
        for di in range(-n, n + 1):
            src = f[max(0, -dj):ny - max(0, dj), max(0, -di):nx - max(0, di)]
            out[max(0, dj):ny - max(0, -dj), max(0, di):nx - max(0, -di)] |= src
    return out


def _split_positions(lo, hi, min_len):
    return range(lo + min_len, hi - min_len + 1)


def _cluster_box(F, box, min_len, max_len, eff, out):
    i0, j0, i1, j1 = box
    sub = F[j0:j1, i0:i1]
    if not sub.any():
        return
    js, is_ = np.nonzero(sub)
    t = [i0 + int(is_.min()), j0 + int(js.min()), i0 + int(is_.max()) + 1, j0 + int(js.max()) + 1]
    # grow to min_len inside the box: upper side first
    for d in (0, 1):
        lo, hi = t[d], t[d + 2]
        blo, bhi = box[d], box[d + 2]
        need = min_len - (hi - lo)
        if need > 0:
            up = min(need, bhi - hi)
            hi += up
            need -= up
            lo -= min(need, lo - blo)
        t[d], t[d + 2] = lo, hi
    ti0, tj0, ti1, tj1 = t
    T = F[tj0:tj1, ti0:ti1]
    w, h = ti1 - ti0, tj1 - tj0
    nflag = int(T.sum())
    if nflag >= eff * w * h and w <= max_len and h <= max_len:
        out.append((ti0, tj0, ti1, tj1))
        return
    order = (0, 1) if w >= h else (1, 0)
    sig = {0: T.sum(axis=0), 1: T.sum(axis=1)}  # x: per column, y: per row
    lo_of = {0: ti0, 1: tj0}
    hi_of = {0: ti1, 1: tj1}
    split = None
    # (a) holes
    for d in order:
        S, lo, hi = sig[d], lo_of[d], hi_of[d]
        for p in _split_positions(lo, hi, min_len):
            if S[p - lo] == 0:
                split = (d, p)
                break
        if split:
            break
    # (b) strongest sign change of the second difference
    if split is None:
        best = None
        for rank, d in enumerate(order):
            S, lo, hi = sig[d].astype(np.int64), lo_of[d], hi_of[d]
            n = hi - lo
            if n < 4:
                continue
            lap = S[:-2] - 2 * S[1:-1] + S[2:]  # lap[k - 1] at slice k, k = 1 .. n-2
            for k in range(1, n - 2):
                a, b = lap[k - 1], lap[k]
                p = lo + k + 1
                if a * b < 0 and lo + min_len <= p <= hi - min_len:
                    key = (-abs(int(b - a)), rank, p)
                    if best is None or key < best[0]:
                        best = (key, d, p)
        if best is not None:
            split = (best[1], best[2])
    # (c) bisect the longer side
    if split is None:
        for d in order:
            lo, hi = lo_of[d], hi_of[d]
            p = lo + (hi - lo) // 2
            if p - lo >= min_len and hi - p >= min_len:
                split = (d, p)
                break
    if split is None:
        out.append((ti0, tj0, ti1, tj1))
        return
    d, p = split
    if d == 0:
        _cluster_box(F, (ti0, tj0, p, tj1), min_len, max_len, eff, out)
        _cluster_box(F, (p, tj0, ti1, tj1), min_len, max_len, eff, out)
    else:
        _cluster_box(F, (ti0, tj0, ti1, p), min_len, max_len, eff, out)
        _cluster_box(F, (ti0, p, ti1, tj1), min_len, max_len, eff, out)


def regions(level: int, nx: int, ny: int, patches, n_nest: int = 2):
    """Regions where patches of level + 1 may be placed (level cell indices)."""
    if level == 0:
        return [(0, 0, nx, ny)]
    out = []
    for (i0, j0, i1, j1) in patches:
        a0 = i0 if i0 == 0 else i0 + n_nest
        b0 = j0 if j0 == 0 else j0 + n_nest
        a1 = i1 if i1 == nx else i1 - n_nest
        b1 = j1 if j1 == ny else j1 - n_nest
        if a1 > a0 and b1 > b0:
            out.append((a0, b0, a1, b1))
    return out


def cluster(flags: np.ndarray, level: int, patches, r: int, n_buf: int, eff: float, min_side: int,
            max_side: int, n_nest: int = 2):
    """Boxes of level + 1 (fine indices, sorted by (j0, i0)) covering the dilated flags of
    `level` inside the nesting regions."""
    ny, nx = flags.shape
    F = dilate(flags, n_buf)
    min_len = -(-min_side // r)
    max_len = max_side // r
    boxes = []
    for R in regions(level, nx, ny, patches, n_nest):
        mask = np.zeros_like(F)
        i0, j0, i1, j1 = R
        mask[j0:j1, i0:i1] = F[j0:j1, i0:i1]
        _cluster_box(mask, R, min_len, max_len, eff, boxes)
    boxes.sort(key=lambda b: (b[1], b[0]))
    return [(b[0] * r, b[1] * r, b[2] * r, b[3] * r) for b in boxes]
