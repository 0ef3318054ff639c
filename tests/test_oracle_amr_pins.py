"""Pins of the oracle's AMR pieces against what the paper and the mathematics fix.

Refinement (Sec. 2.1): interpolating eta_m (not h_m) with minmod slopes keeps the
mean of every coarse cell (so mass away from the shore), creates no new extrema,
reproduces linear surfaces exactly and reduces to the one-layer scheme. Coarsening
(Sec. 2.2, Eq. (11)) is the mean of the fine cells of every component. Flags are the
gradient test of the top surface; clustering boxes cover every buffered flag, are
disjoint, nested and within the side bounds. The composite AMR solution conserves
layer masses on walled wet domains and keeps a lake at rest.
"""
import itertools

import numpy as np
import pytest

import oracle as O
from oracle import cluster as C
from oracle.amr import OracleAMR
from paper_1803_01450_gb300 import inputs as I


def _coarse_setup(seed, M=2, n=12, r=4, wet=True):
    rng = np.random.default_rng(seed)
    Bf = -10.0 + 0.3 * rng.standard_normal((n * r, n * r))
    Bc = O.bathy_average(Bf, r)
    eta2 = -4.0 + 0.2 * rng.standard_normal((n, n))
    eta1 = 0.0 + 0.2 * rng.standard_normal((n, n))
    q = np.zeros((3 * M, n, n))
    if M == 3:
        eta3 = -7.0 + 0.2 * rng.standard_normal((n, n))
        q[6] = eta3 - Bc
        q[3] = eta2 - eta3
        q[0] = eta1 - eta2
    elif M == 2:
        q[3] = eta2 - Bc
        q[0] = eta1 - eta2
    else:
        q[0] = eta1 - Bc
    for m in range(M):
        q[3 * m + 1] = 0.3 * rng.standard_normal((n, n)) * q[3 * m]
        q[3 * m + 2] = 0.3 * rng.standard_normal((n, n)) * q[3 * m]
    return q, Bc, Bf


def _interp_all(P, q, Bc, Bf, r):
    qp, Bp = O.pad(q, Bc)
    O.fill_walls(P.M, qp, Bp)
    n = q.shape[1]
    return O.interp_fine(P, r, qp, Bp, (0, 0, n, n), Bf)


@pytest.mark.parametrize("M", [1, 2, 3])
@pytest.mark.parametrize("r", [2, 4])
def test_refinement_preserves_cell_means(M, r):
    """Sec. 2.1: the offsets (a + 1/2)/r - 1/2 sum to zero, so the fine surfaces average to
    the coarse surface; with B averaged by the same operator and no clipping, the fine
    depths average to the coarse depth (mass is conserved away from the shore)."""
    P = O.params(M=M, dry_tol=1e-6)
    q, Bc, Bf = _coarse_setup(1, M=M, r=r)
    fine = _interp_all(P, q, Bc, Bf, r)
    for m in range(M):
        avg = O.average_coarse(fine[3 * m], r)
        assert np.abs(avg - q[3 * m]).max() <= 1e-13 * np.abs(q[3 * m]).max()
        for k in (1, 2):
            avg = O.average_coarse(fine[3 * m + k], r)
            assert np.abs(avg - q[3 * m + k]).max() <= 1e-13 * np.abs(q[3 * m + k]).max()


@pytest.mark.parametrize("r", [2, 4])
def test_refinement_no_new_extrema(r):
    """Sec. 2.1 (minmod, Eq. (10)): every fine surface value lies within the range of the
    coarse cell and its face neighbours."""
    P = O.params(M=2, dry_tol=1e-6)
    q, Bc, Bf = _coarse_setup(2, r=r)
    fine = _interp_all(P, q, Bc, Bf, r)
    n = q.shape[1]
    eta_c = [Bc + q[3] + q[0], Bc + q[3]]
    Bf_eta = [Bf + fine[3] + fine[0], Bf + fine[3]]
    for m in range(2):
        e = np.pad(eta_c[m], 1, mode="edge")
        lo = np.minimum.reduce([e[1:-1, 1:-1], e[1:-1, :-2], e[1:-1, 2:], e[:-2, 1:-1], e[2:, 1:-1]])
        hi = np.maximum.reduce([e[1:-1, 1:-1], e[1:-1, :-2], e[1:-1, 2:], e[:-2, 1:-1], e[2:, 1:-1]])
        ef = Bf_eta[m].reshape(n, r, n, r)
        tol = 1e-12 * np.abs(eta_c[m]).max()
        assert np.all(ef >= lo[:, None, :, None] - tol)
        assert np.all(ef <= hi[:, None, :, None] + tol)


@pytest.mark.parametrize("r", [2, 4])
def test_refinement_reproduces_linear_surfaces(r):
    """minmod of two equal differences is that difference: linear surfaces are refined
    exactly (the offsets are exact binary fractions for r = 2, 4)."""
    P = O.params(M=2, dry_tol=1e-6)
    n = 10
    x = np.arange(n) + 0.5
    X, Y = np.meshgrid(x, x)
    Bc = -20.0 * np.ones((n, n))
    Bf = -20.0 * np.ones((n * r, n * r))
    eta2 = -8.0 + 0.25 * X - 0.125 * Y
    eta1 = 0.5 + 0.0625 * X + 0.5 * Y
    q = np.zeros((6, n, n))
    q[3] = eta2 - Bc
    q[0] = eta1 - eta2
    fine = _interp_all(P, q, Bc, Bf, r)
    xf = (np.arange(n * r) + 0.5) / r
    XF, YF = np.meshgrid(xf, xf)
    sl = slice(r, -r)  # interior coarse cells (the walls flatten the boundary slopes)
    assert np.abs((Bf + fine[3])[sl, sl] - (-8.0 + 0.25 * XF - 0.125 * YF)[sl, sl]).max() <= 1e-13
    assert np.abs((Bf + fine[3] + fine[0])[sl, sl] - (0.5 + 0.0625 * XF + 0.5 * YF)[sl, sl]).max() <= 1e-13


def test_refinement_two_layers_reduce_to_one():
    """With the lower layer absent (h_2 = 0), refining two layers equals refining one."""
    P1, P2 = O.params(M=1, dry_tol=1e-6), O.params(M=2, dry_tol=1e-6)
    q1, Bc, Bf = _coarse_setup(3, M=1)
    q2 = np.zeros((6,) + q1.shape[1:])
    q2[:3] = q1
    f1 = _interp_all(P1, q1, Bc, Bf, 4)
    f2 = _interp_all(P2, q2, Bc, Bf, 4)
    assert np.array_equal(f1, f2[:3])
    assert not f2[3:].any()


def test_coarsening_is_block_mean_and_round_trip():
    """Sec. 2.2, Eq. (11) in 2-D: the block mean of every component (numpy reshape mean
    as the reference); coarsening a refinement returns the coarse state."""
    rng = np.random.default_rng(5)
    qf = rng.standard_normal((6, 24, 36))
    avg = O.average_coarse(qf, 4)
    ref = qf.reshape(6, 6, 4, 9, 4).mean(axis=(2, 4))
    assert np.abs(avg - ref).max() <= 1e-15 * np.abs(ref).max() * 16
    P = O.params(M=2, dry_tol=1e-6)
    q, Bc, Bf = _coarse_setup(6, r=4)
    back = O.average_coarse(_interp_all(P, q, Bc, Bf, 4), 4)
    assert np.abs(back - q).max(axis=(1, 2)).max() <= 1e-13 * np.abs(q).max()


def test_bathymetry_levels_are_block_means():
    rng = np.random.default_rng(9)
    Bf = rng.standard_normal((32, 48))
    assert np.allclose(O.bathy_average(Bf, 4), Bf.reshape(8, 4, 12, 4).mean(axis=(1, 3)), rtol=1e-14, atol=1e-15)


def test_flags_match_numpy_gradient():
    """Flags of |grad eta_1| > tol on a fully wet level equal numpy.gradient's central /
    one-sided differences (evaluated with a margin around the threshold)."""
    w = I.small(50)
    q, B = w["q"], w["B"]
    dx = w["dx"]
    tol = 1e-3
    fl = O.flags(2, q, B, np.ones((50, 50), np.uint8), 1e-6, dx, dx, tol)
    eta = B + q[3] + q[0]
    gy, gx = np.gradient(eta, dx, dx)
    g2 = gx * gx + gy * gy
    clear = np.abs(g2 - tol * tol) > 1e-9 * tol * tol
    assert np.array_equal(fl[clear].astype(bool), (g2 > tol * tol)[clear])
    assert fl.sum() > 50


def _check_boxes(flags, level, patches, r, n_buf, eff, min_side, max_side, boxes, n_nest=2):
    ny, nx = flags.shape
    F = C.dilate(flags, n_buf)
    regs = C.regions(level, nx, ny, patches, n_nest)
    allowed = np.zeros_like(F)
    for (i0, j0, i1, j1) in regs:
        allowed[j0:j1, i0:i1] = True
    need = F & allowed
    cov = np.zeros((ny, nx), int)
    for (a, b, c, d) in boxes:
        assert a % r == 0 and b % r == 0 and c % r == 0 and d % r == 0
        ci0, cj0, ci1, cj1 = a // r, b // r, c // r, d // r
        assert ci1 - ci0 <= max_side // r and cj1 - cj0 <= max_side // r
        assert any(ci0 >= R[0] and cj0 >= R[1] and ci1 <= R[2] and cj1 <= R[3] for R in regs)
        cov[cj0:cj1, ci0:ci1] += 1
    assert cov.max() <= 1, "boxes overlap"
    assert np.all(cov[need] == 1), "a buffered flag is not covered"


def test_dilation_brute_force():
    rng = np.random.default_rng(11)
    f = rng.random((9, 11)) < 0.1
    d = C.dilate(f, 2)
    for j, i in itertools.product(range(9), range(11)):
        ref = f[max(0, j - 2):j + 3, max(0, i - 2):i + 3].any()
        assert d[j, i] == ref


@pytest.mark.parametrize("seed", range(12))
def test_clustering_invariants_random(seed):
    rng = np.random.default_rng(seed)
    nx, ny = int(rng.integers(20, 70)), int(rng.integers(20, 70))
    flags = np.zeros((ny, nx), bool)
    for _ in range(int(rng.integers(1, 5))):
        cx, cy, rad = rng.integers(0, nx), rng.integers(0, ny), rng.integers(2, 9)
        Y, X = np.mgrid[0:ny, 0:nx]
        flags |= (X - cx) ** 2 + (Y - cy) ** 2 < rad ** 2
    flags &= rng.random((ny, nx)) < 0.8
    boxes = C.cluster(flags, 0, [(0, 0, nx, ny)], 4, 2, 0.7, 16, 64)
    _check_boxes(flags, 0, [(0, 0, nx, ny)], 4, 2, 0.7, 16, 64, boxes)
    # refined level: regions are shrunk patches
    patches = [(0, 0, nx // 2, ny), (nx // 2, 0, nx, ny // 2)]
    boxes = C.cluster(flags, 1, patches, 4, 2, 0.7, 16, 64)
    _check_boxes(flags, 1, patches, 4, 2, 0.7, 16, 64, boxes)


def test_clustering_tiny_exhaustive():
    """Every 4x4 flag pattern (65536 of them) on an 8x8 region with r = 2, min side 2 fine
    cells: covering, disjoint, inside, efficiency or unsplittable."""
    nx = ny = 8
    for bits in range(0, 1 << 16, 7):
        f = np.zeros((ny, nx), bool)
        sub = np.array([(bits >> k) & 1 for k in range(16)], bool).reshape(4, 4)
        f[2:6, 2:6] = sub
        boxes = C.cluster(f, 0, [(0, 0, nx, ny)], 2, 0, 0.7, 2, 16)
        _check_boxes(f, 0, [(0, 0, nx, ny)], 2, 0, 0.7, 2, 16, boxes)


# ------------------------------------------------------------------ composite AMR
@pytest.mark.parametrize("unsplit", [0, 1])
def test_amr_mass_conservation_with_reflux(unsplit):
    """Walled, wet, flat-bottom two-layer AMR run: the composite mass of each layer is
    constant to rounding (the reflux makes the coarse/fine edges conservative; in the unsplit
    form the recorded fluxes carry the transverse corrections, and sibling patches compute
    their shared edges from the same cells)."""
    w = I.small(50)
    P = O.params(M=2, dry_tol=1e-6, unsplit=unsplit)
    A = OracleAMR(P, (0, 0, 1, 1), 50, 50, 2, [2], -np.ones((100, 100)), min_side=16, max_side=64)
    A.set_state(0, w["q"])
    m0 = A.mass()
    A.advance(12, regrid_interval=4)
    m1 = A.mass()
    assert len(A.lev[1].patches) > 0
    assert np.all(np.abs(m1 - m0) <= 1e-13 * m0)


@pytest.mark.parametrize("unsplit", [0, 1])
def test_amr_lake_at_rest_on_shelf(unsplit):
    """Three levels over a shelf at rest: surfaces stay flat, momenta stay zero."""
    n0, r = 16, [2, 2]
    nf = n0 * 4
    Bf = I.shelf_B(np.meshgrid(I.centers(0, 1e5, nf), I.centers(0, 1e5, nf))[0])
    P = O.params(M=2, dry_tol=1e-3, unsplit=unsplit)
    A = OracleAMR(P, (0, 0, 1e5, 1e5), n0, n0, 3, r, Bf, min_side=8, max_side=32)
    q0 = I.layered_state(A.lev[0].B, np.zeros_like(A.lev[0].B), -200.0 * np.ones_like(A.lev[0].B))
    A.set_state(0, q0)
    A.set_patches(1, [(8, 8, 24, 24)])
    A.interp_into(0, A.lev[0].q, A.lev[1].in_patch_mask())
    A.set_patches(2, [(24, 24, 40, 40)])
    A.interp_into(1, A.lev[1].q, A.lev[2].in_patch_mask())
    A.advance(4, dt=2.0)
    for l, V in enumerate(A.lev):
        m = V.in_patch_mask() if l else np.ones((V.ny, V.nx), bool)
        eta1 = V.B + V.q[3] + V.q[0]
        assert np.abs(eta1[m]).max() <= 1e-13 * 4000
        assert np.abs(V.q[[1, 2, 4, 5]][:, m]).max() <= 1e-13 * 4000


def _shallow_region_amr(dynamic, n=32, r=4, steps=12):
    """Two levels over a basin that is deep (-1) in the west and shallow (-0.05) in the east,
    a hump in the shallow part: the refined patches sit where the waves are slow."""
    P = O.params(M=2, rho=(1000.0, 1025.0), dry_tol=1e-6)
    nf = n * r
    xf = (np.arange(nf) + 0.5) / nf
    Xf, _ = np.meshgrid(xf, xf)
    Bf = np.where(Xf < 0.5, -1.0, -0.05)
    A = OracleAMR(P, (0, 0, 1, 1), n, n, 2, [r], Bf, flag_tol=2e-3, min_side=8, max_side=32, dynamic_rt=dynamic)
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x)
    B0 = O.bathy_average(Bf, r)
    eta1 = 0.004 * np.exp(-((X - 0.75) ** 2 + (Y - 0.5) ** 2) / 0.004)
    q = np.zeros((6, n, n))
    q[3] = np.maximum(-0.02 - B0, 0.0)
    q[0] = eta1 - np.maximum(-0.02, B0)
    A.set_state(0, q)
    return A, steps


def test_dynamic_time_ratio_rule_values():
    """The rule on constructed rates: the fewest substeps with dt_parent / r_t * rate <= cfl,
    clamped to [1, r]; an exact multiple does not take an extra substep; the first step after
    a regrid, a level without speeds and the fixed choice take r."""
    A, _ = _shallow_region_amr(True)
    A.cfl = 0.5
    for rate, dtp, want in ((10.0, 0.2, 4), (10.0, 0.1, 2), (10.0, 0.05, 1), (10.0, 0.075, 2),
                            (1.0, 0.01, 1), (1000.0, 0.2, 4), (10.0, 0.15, 3)):
        A.rates[1] = rate
        assert A.time_ratio(1, dtp) == want, (rate, dtp)
    A.rates[1] = 1.0
    A.fresh = True
    assert A.time_ratio(1, 0.01) == 4
    A.fresh = False
    A.rates[1] = 0.0
    assert A.time_ratio(1, 0.01) == 4
    A.dynamic_rt = False
    A.rates[1] = 1.0
    assert A.time_ratio(1, 0.01) == 4


def test_dynamic_time_ratio_takes_fewer_fine_steps_within_cfl():
    """Sec. 2: with refined patches only in shallow water the fine level needs fewer steps
    per coarse step than the spatial ratio; every step of every level keeps its Courant
    number at cfl (to the change of the speeds from one step to the next)."""
    A, steps = _shallow_region_amr(True)
    courant = []
    taken = []
    orig = A.step_level

    def record(l, dt, alpha):
        orig(l, dt, alpha)
        taken.append((l, dt))

    A.step_level = record
    for k in range(steps):
        taken.clear()
        A.advance(1, regrid_interval=4 if k % 4 == 0 else 0)
        for l in range(A.L):
            dts = [d for (ll, d) in taken if ll == l]
            if dts:
                V = A.lev[l]
                courant.append(max(dts) * max(A.smax[l][0] / V.dx, A.smax[l][1] / V.dy))
    assert A.level_steps[0] == steps
    assert 0 < A.level_steps[1] < 4 * steps  # fewer than the fixed ratio's
    assert max(courant) <= A.cfl * (1 + 1e-3), max(courant)
    assert min(courant[1::2]) < 0.5 * A.cfl  # a first step after a regrid took the fixed ratio


def test_dynamic_time_ratio_conserves_mass_and_rest():
    A, steps = _shallow_region_amr(True)
    A.advance(1, regrid_interval=4)
    m0 = A.mass()
    A.advance(steps, regrid_interval=4)
    assert np.all(np.abs(A.mass() - m0) <= 1e-13 * np.abs(m0))
    # lake at rest stays at rest with dynamic ratios
    P = O.params(M=2, rho=(1000.0, 1025.0), dry_tol=1e-6)
    n, r = 24, 2
    nf = n * r
    xf = (np.arange(nf) + 0.5) / nf
    Xf, Yf = np.meshgrid(xf, xf)
    # a bump that keeps both layers wet (averaging across an internal shoreline, where a layer
    # ends inside a coarse cell, does not keep the rest state: Sec. 2.2 holds away from shores)
    Bf = -1.0 + 0.25 * np.exp(-((Xf - 0.6) ** 2 + (Yf - 0.5) ** 2) / 0.01)
    R = OracleAMR(P, (0, 0, 1, 1), n, n, 2, [r], Bf, flag_tol=1e-9, min_side=8, max_side=32, dynamic_rt=True)
    B0 = O.bathy_average(Bf, r)
    q = np.zeros((6, n, n))
    q[3] = np.maximum(-0.6 - B0, 0.0)
    q[0] = 0.0 - np.maximum(-0.6, B0)
    R.set_state(0, q)
    R.set_patches(1, [(16, 16, 32, 32)])
    R.interp_into(0, R.lev[0].q, R.lev[1].in_patch_mask())
    R.advance(6)
    assert np.abs(R.lev[0].q[[1, 2, 4, 5]]).max() <= 1e-13


def _golden_refinement():
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "refinement_worked_examples.json")) as f:
        return json.load(f)


def test_refinement_worked_examples():
    """The hand-worked refinement examples of tests/golden (Sec. 2.1 Eqs. (4), (5), (10), the
    bottom-up layer loop and the clipping at zero depth) reproduced by the oracle."""
    P = O.params(M=2, dry_tol=1e-6)
    for ex in _golden_refinement()["examples"]:
        c = ex["coarse"]
        q = np.zeros((6, 1, 3))
        q[0, 0], q[1, 0] = c["h1"], c["hu1"]
        q[3, 0], q[4, 0] = c["h2"], c["hu2"]
        B = np.array([c["B"]], float)
        qp, Bp = O.pad(q, B)
        O.fill_walls(2, qp, Bp)
        Bf = np.array([ex["fine_B"], ex["fine_B"]], float)
        out = O.interp_fine(P, 2, qp, Bp, (1, 0, 2, 1), Bf)
        f = ex["fine"]
        for name, field in (("h1", 0), ("hu1", 1), ("h2", 3), ("hu2", 4)):
            for row in range(2):
                assert np.allclose(out[field, row], f[name], rtol=1e-14, atol=1e-14), (ex["name"], name, out[field])
        assert not out[[2, 5]].any()
