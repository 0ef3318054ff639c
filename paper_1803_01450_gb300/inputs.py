"""Seeded synthetic workloads shaped like the paper's demonstration.

This module only draws random numbers and lays out initial data (bathymetry,
layer interfaces, Gaussian surface humps). It contains none of the solver's
arithmetic; both the CUDA library's tests/benchmark and the CPU oracle take
their inputs from here so that both see bit-identical arrays.

The paper's own setup (a plane wave running from deep water onto a
discontinuous shelf, depth scaled to -1, Sec. 3) is not available, so the
workloads below stand in for it:

* ``small``: [0,1]^2, 50x50 coarse cells, flat B = -1, interface at -0.6, one
  Gaussian hump of amplitude 0.02 on the free surface (two layers, walls).
* ``scale``: [0,100 km]^2, 2048x2048 fixed grid, shelf bathymetry
  B(x) = -4000 + 3800 sigmoid((x - 70 km) / 5 km), interface at -200 m, eight
  seeded humps (amplitude U[0.5,2] m, width U[2,10] km).
* ``shore``: the shelf above, rising linearly from x = 95 km to +20 m at the
  east wall, so both layers meet a dry shore.
* ``adjoint``: 512x512, B = -4000 + 500 sin(2 pi x/L) cos(2 pi y/L).
* ``ensemble``: per member a seeded domain size, shelf depth and position and
  1-4 humps.

Seeds are ``config_index * 1000 + member`` (numpy PCG64).
"""
from __future__ import annotations

import math

import numpy as np

G = 9.81
RHO = (1000.0, 1025.0)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def centers(x0: float, x1: float, n: int) -> np.ndarray:
    dx = (x1 - x0) / n
    return x0 + (np.arange(n) + 0.5) * dx


def humps(seed: int, n: int, L: float = 1e5, amp=(0.5, 2.0), width=(2e3, 1e4),
          xr=(1e4, 6e4), yr=(1e4, 9e4)):
    """Gaussian hump parameters (A, w, xc, yc) drawn in a fixed order."""
    g = rng(seed)
    A = g.uniform(amp[0], amp[1], n)
    w = g.uniform(width[0], width[1], n)
    xc = g.uniform(xr[0], xr[1], n)
    yc = g.uniform(yr[0], yr[1], n)
    return A, w, xc, yc


def hump_field(X, Y, A, w, xc, yc):
    out = np.zeros_like(X)
    for a, ww, x0, y0 in zip(A, w, xc, yc):
        out += a * np.exp(-((X - x0) ** 2 + (Y - y0) ** 2) / ww ** 2)
    return out


def shelf_B(x, depth=4000.0, shelf_x=7e4, shelf_top=200.0, scale=5e3):
    return -depth + (depth - shelf_top) * (1.0 / (1.0 + np.exp(-(x - shelf_x) / scale)))


def shore_B(x, **kw):
    """Shelf, then a straight ramp from its value at 95 km to +20 m at 100 km."""
    b = shelf_B(x, **kw)
    b95 = shelf_B(np.array([9.5e4]), **kw)[0]
    ramp = b95 + (20.0 - b95) * (x - 9.5e4) / 5e3
    return np.where(x <= 9.5e4, b, ramp)


def layered_state(B, eta1, eta2):
    """Conserved fields [6][ny][nx] of a two-layer fluid at rest with surfaces eta1 over eta2.

    A layer absent where the ground is above its lower surface gets depth 0."""
    h2 = np.maximum(0.0, eta2 - B)
    base = np.maximum(B, eta2)
    h1 = np.maximum(0.0, eta1 - base)
    z = np.zeros_like(B)
    return np.stack([h1, z, z.copy(), h2, z.copy(), z.copy()])


def stacked_state(B, etas):
    """Conserved fields [3M][ny][nx] of M layers at rest whose upper surfaces are etas (top
    layer first) above the ground B. A layer absent where the ground or the layers below
    reach above its surface gets depth 0."""
    M = len(etas)
    q = np.zeros((3 * M,) + np.shape(B))
    lower = np.asarray(B, dtype=float)
    for m in range(M - 1, -1, -1):
        top = np.maximum(np.broadcast_to(etas[m], lower.shape), lower)
        q[3 * m] = top - lower
        lower = top
    return q


def shore3(n: int, seed: int = 3000, L: float = 1e5, n_humps: int = 8):
    """Three-layer shore workload on an n x n grid: surfaces humps / -50 m / -200 m over the
    shore bathymetry, so both lower layers meet the rising ground before the top one."""
    x = centers(0.0, L, n)
    X, Y = np.meshgrid(x, x)
    B = shore_B(X)
    A, w, xc, yc = humps(seed, n_humps, L)
    eta1 = hump_field(X, Y, A, w, xc, yc)
    q = stacked_state(B, (eta1, -50.0 + 0.0 * X, -200.0 + 0.0 * X))
    return dict(q=q, B=B, dx=L / n, dy=L / n, domain=(0.0, 0.0, L, L), dry_tol=1e-3)


def shore4(n: int, seed: int = 3000, L: float = 1e5, n_humps: int = 8):
    """Four-layer shore workload on an n x n grid: surfaces humps / -50 m / -120 m / -250 m
    over the shore bathymetry, so the lower layers meet the rising ground one after another."""
    x = centers(0.0, L, n)
    X, Y = np.meshgrid(x, x)
    B = shore_B(X)
    A, w, xc, yc = humps(seed, n_humps, L)
    eta1 = hump_field(X, Y, A, w, xc, yc)
    q = stacked_state(B, (eta1, -50.0 + 0.0 * X, -120.0 + 0.0 * X, -250.0 + 0.0 * X))
    return dict(q=q, B=B, dx=L / n, dy=L / n, domain=(0.0, 0.0, L, L), dry_tol=1e-3)


def scale4(n: int = 2048, seed: int = 1000, L: float = 1e5):
    """Four-layer version of the scale workload: the same shelf and humps, surfaces
    humps / -100 m / -300 m / -600 m (the lower layers end where the shelf rises above them)."""
    x = centers(0.0, L, n)
    X, Y = np.meshgrid(x, x)
    B = shelf_B(X)
    A, w, xc, yc = humps(seed, 8, L)
    eta1 = hump_field(X, Y, A, w, xc, yc)
    q = stacked_state(B, (eta1, -100.0 + 0.0 * X, -300.0 + 0.0 * X, -600.0 + 0.0 * X))
    return dict(q=q, B=B, dx=L / n, dy=L / n, domain=(0.0, 0.0, L, L), dry_tol=1e-3)


def small(n: int = 50):
    x = centers(0.0, 1.0, n)
    X, Y = np.meshgrid(x, x)
    B = -np.ones((n, n))
    eta1 = 0.02 * np.exp(-((X - 0.3) ** 2 + (Y - 0.5) ** 2) / 0.005)
    q = layered_state(B, eta1, -0.6 * np.ones_like(B))
    return dict(q=q, B=B, dx=1.0 / n, dy=1.0 / n, domain=(0.0, 0.0, 1.0, 1.0), dry_tol=1e-6)


def small_B(n: int):
    return -np.ones((n, n))


def scale(n: int = 2048, seed: int = 1000, L: float = 1e5):
    x = centers(0.0, L, n)
    X, Y = np.meshgrid(x, x)
    B = shelf_B(X)
    A, w, xc, yc = humps(seed, 8, L)
    eta1 = hump_field(X, Y, A, w, xc, yc)
    q = layered_state(B, eta1, -200.0 * np.ones_like(B))
    return dict(q=q, B=B, dx=L / n, dy=L / n, domain=(0.0, 0.0, L, L), dry_tol=1e-3)


def scale3(n: int = 2048, seed: int = 1000, L: float = 1e5):
    """Three-layer version of the scale workload: the same shelf and humps, surfaces
    humps / -100 m / -600 m (the bottom layer ends where the shelf rises above -600 m)."""
    x = centers(0.0, L, n)
    X, Y = np.meshgrid(x, x)
    B = shelf_B(X)
    A, w, xc, yc = humps(seed, 8, L)
    eta1 = hump_field(X, Y, A, w, xc, yc)
    q = stacked_state(B, (eta1, -100.0 + 0.0 * X, -600.0 + 0.0 * X))
    return dict(q=q, B=B, dx=L / n, dy=L / n, domain=(0.0, 0.0, L, L), dry_tol=1e-3)


def shore_bathymetry(nx: int, ny: int, L: float = 1e5):
    x = centers(0.0, L, nx)
    y = centers(0.0, L, ny)
    X, _ = np.meshgrid(x, y)
    return shore_B(X)


def shore(n: int, seed: int = 3000, L: float = 1e5, n_humps: int = 8):
    """Shore workload on an n x n grid (B sampled at this grid's cell centres)."""
    x = centers(0.0, L, n)
    X, Y = np.meshgrid(x, x)
    B = shore_B(X)
    A, w, xc, yc = humps(seed, n_humps, L)
    eta1 = hump_field(X, Y, A, w, xc, yc)
    q = layered_state(B, eta1, -200.0 * np.ones_like(B))
    return dict(q=q, B=B, dx=L / n, dy=L / n, domain=(0.0, 0.0, L, L), dry_tol=1e-3)


def adjoint_bathymetry(n: int = 512, L: float = 1e5):
    x = centers(0.0, L, n)
    X, Y = np.meshgrid(x, x)
    return -4000.0 + 500.0 * np.sin(2 * math.pi * X / L) * np.cos(2 * math.pi * Y / L)


def adjoint_eta1(n: int = 512, seed: int = 4000, L: float = 1e5):
    x = centers(0.0, L, n)
    X, Y = np.meshgrid(x, x)
    A, w, xc, yc = humps(seed, 8, L)
    return hump_field(X, Y, A, w, xc, yc)


def gauge_cells(n: int, n_gauges: int = 32, seed: int = 4100):
    """Seeded interior gauge cells (i, j), 1 <= i, j <= n - 2."""
    g = rng(seed)
    return np.stack([g.integers(1, n - 1, n_gauges), g.integers(1, n - 1, n_gauges)], axis=1).astype(np.int32)


def ensemble_member(k: int, seed_base: int = 5000, L: float = 1e5, n_min: int = 128, n_max: int = 512):
    """One member of the ensemble workload: its coarse size and initial data."""
    g = rng(seed_base + k)
    n = int(g.integers(n_min, n_max + 1))
    depth = g.uniform(3000.0, 5000.0)
    sx = g.uniform(6e4, 8e4)
    nh = int(g.integers(1, 5))
    A = g.uniform(0.5, 2.0, nh)
    w = g.uniform(2e3, 1e4, nh)
    xc = g.uniform(1e4, 6e4, nh)
    yc = g.uniform(1e4, 9e4, nh)
    return dict(n=n, depth=depth, shelf_x=sx, humps=(A, w, xc, yc), L=L)


def ensemble_state(member: dict, n: int):
    """Initial data of an ensemble member on an n x n grid."""
    L = member["L"]
    x = centers(0.0, L, n)
    X, Y = np.meshgrid(x, x)
    B = shelf_B(X, depth=member["depth"], shelf_x=member["shelf_x"])
    eta1 = hump_field(X, Y, *member["humps"])
    q = layered_state(B, eta1, -200.0 * np.ones_like(B))
    return q, B


def random_layout(seed: int, nx: int, ny: int, n_boxes: int, r: int, side=(16, 64), parents=None,
                  margin: int = 2, max_tries: int = 200000):
    """Seeded random non-overlapping patch boxes of one refined level (fine indices,
    half-open (i0, j0, i1, j1)), sides drawn from U{side} rounded to multiples of r, corners
    on multiples of r. With `parents` (boxes of the coarser level, its indices) every box
    lies inside one parent shrunk by `margin` coarse cells (not at the domain boundary).
    Stands in for the patch layouts of a regridded level; returns fewer boxes than asked
    when no more fit."""
    g = rng(seed)
    occ = np.zeros((ny // r, nx // r), dtype=bool)
    boxes = []
    regions = [(0, 0, nx // r, ny // r)]
    if parents is not None:
        NXc, NYc = nx // r, ny // r
        regions = []
        for (i0, j0, i1, j1) in parents:
            a0 = i0 if i0 == 0 else i0 + margin
            b0 = j0 if j0 == 0 else j0 + margin
            a1 = i1 if i1 == NXc else i1 - margin
            b1 = j1 if j1 == NYc else j1 - margin
            if a1 > a0 and b1 > b0:
                regions.append((a0, b0, a1, b1))
    tries = 0
    while len(boxes) < n_boxes and tries < max_tries:
        tries += 1
        a0, b0, a1, b1 = regions[int(g.integers(0, len(regions)))]
        w = max(1, int(g.integers(side[0], side[1] + 1)) // r)
        h = max(1, int(g.integers(side[0], side[1] + 1)) // r)
        w, h = min(w, a1 - a0), min(h, b1 - b0)
        if w <= 0 or h <= 0:
            continue
        i0 = int(g.integers(a0, a1 - w + 1))
        j0 = int(g.integers(b0, b1 - h + 1))
        if occ[j0:j0 + h, i0:i0 + w].any():
            continue
        occ[j0:j0 + h, i0:i0 + w] = True
        boxes.append((i0 * r, j0 * r, (i0 + w) * r, (j0 + h) * r))
    boxes.sort(key=lambda b: (b[1], b[0]))
    return boxes


def gaussian_random_state(seed: int, M: int, nx: int, ny: int, depth=(1.0, 0.5), amp=0.05, vel=0.05):
    """Random smooth-ish wet state for parity tests: positive depths with perturbations
    and small velocities; bathymetry with gentle variation."""
    g = rng(seed)
    B = -sum(depth) + 0.1 * g.standard_normal((ny, nx)).cumsum(axis=1) / max(nx, 1) ** 0.5
    q = np.zeros((3 * M, ny, nx))
    eta_prev = None
    for m in range(M - 1, -1, -1):
        h = depth[m] * (1.0 + amp * g.standard_normal((ny, nx)))
        q[3 * m] = np.maximum(h, 0.1 * depth[m])
        q[3 * m + 1] = vel * q[3 * m] * g.standard_normal((ny, nx))
        q[3 * m + 2] = vel * q[3 * m] * g.standard_normal((ny, nx))
    del eta_prev
    return q, B
