"""GPU parity of the unsplit step (transverse Riemann solves, corner-transport form) against
the oracle's unsplit step: fixed walled grids (one and two layers, orders 1 and 2, shapes
that span several tiles with a ragged last one), a shore with dry cells, lake at rest, the
reported Courant number, x/y exchange symmetry on the GPU itself, subcycled AMR runs with
regrids (two and three levels), the dynamic time ratio (members passing substeps through the
update kernel), three layers, and the options the unsplit step does not take. Tolerance: 1e-11 relative
per field, as for the split step (reciprocals, closed-form strengths and fused
multiply-adds against plainly rounded oracle arithmetic)."""
import numpy as np
import pytest

import oracle as O
from oracle.amr import OracleAMR
from paper_1803_01450_gb300 import inputs as I
from conftest import rel_err, report, state_err, state_scale

pytestmark = pytest.mark.gpu
TOL = 1e-11


def _run_both(pkg, q, B, dx, dy, dts, M=2, order=2, limiter=2, dry_tol=1e-6, eigen=0, want_cfl=False):
    ny, nx = B.shape
    cfg = pkg.Config(M=M, order=order, limiter=limiter, dry_tol=dry_tol, eigen=eigen, max_levels=1, unsplit=1)
    H = pkg.Hierarchy(cfg, [(0.0, 0.0, nx * dx, ny * dy, nx, ny)])
    H.set_bathymetry(0, B)
    H.set_state(0, 0, q)
    P = O.params(M=M, dry_tol=dry_tol, order=order, limiter=limiter, eigen=eigen, unsplit=1)
    qo = q.copy()
    cfls = []
    for dt in dts:
        c = H.step_level(0, dt=dt, want_cfl=want_cfl)
        qo, smax, _ = O.step_walled(P, qo, B, dx, dy, dt)
        if want_cfl:
            cfls.append((c[0], dt * max(smax[0] / dx, smax[1] / dy)))
    qg = H.get_state(0, 0)
    H.close()
    return qg, qo, cfls


@pytest.mark.parametrize("M,order,limiter", [(2, 2, 2), (2, 1, 0), (2, 2, 1), (1, 2, 2), (1, 1, 0)])
@pytest.mark.parametrize("shape", [(17, 23), (64, 130), (300, 7)])
def test_random_wet_states(mlswe_lib, M, order, limiter, shape):
    ny, nx = shape
    q, B = I.gaussian_random_state(31 + nx + 7 * ny + M, M, nx, ny)
    dx, dy = 1.0 / nx, 1.3 / ny
    dts = [0.3 * min(dx, dy) / 4.0] * 5
    qg, qo, _ = _run_both(mlswe_lib, q, B, dx, dy, dts, M=M, order=order, limiter=limiter)
    err = rel_err(qg, qo)
    assert err.max() < TOL, err


def test_eigen_guess_only_and_courant_report(mlswe_lib):
    q, B = I.gaussian_random_state(6, 2, 40, 33)
    dts = [0.25 / 40 / 4.0] * 4
    qg, qo, cfls = _run_both(mlswe_lib, q, B, 1 / 40, 1 / 33, dts, eigen=1, want_cfl=True)
    assert rel_err(qg, qo).max() < TOL
    for g, o in cfls:
        assert abs(g - o) <= 1e-12 * o


def test_small_workload_100_steps(mlswe_lib):
    w = I.small(50)
    dts = [0.9 * w["dx"] / 3.2] * 100
    qg, qo, _ = _run_both(mlswe_lib, w["q"], w["B"], w["dx"], w["dy"], dts, dry_tol=w["dry_tol"])
    assert rel_err(qg, qo).max() < TOL


def test_shore_wet_dry(mlswe_lib):
    """Both layers meeting dry land (the per-layer transverse split, walls for a layer):
    every field to 1e-11 of its scale (state_scale: a momentum's scale is at least h_max
    sqrt(g h_max) of its layer, since deep water makes near-rest momentum rounding noise)."""
    w = I.shore(96, seed=3001)
    dts = [0.5 * w["dx"] / 210.0] * 20
    qg, qo, _ = _run_both(mlswe_lib, w["q"], w["B"], w["dx"], w["dy"], dts, dry_tol=w["dry_tol"])
    err = state_err(qg, qo, 2)
    report("unsplit_shore_96_20steps", err)
    assert err.max() < TOL, err


def test_lake_at_rest(mlswe_lib):
    n = 64
    B = I.shore_bathymetry(n, n)
    q = I.layered_state(B, np.zeros_like(B), -200.0 * np.ones_like(B))
    cfg = mlswe_lib.Config(M=2, max_levels=1, unsplit=1)
    H = mlswe_lib.Hierarchy(cfg, [(0.0, 0.0, 1e5, 1e5, n, n)])
    H.set_bathymetry(0, B)
    H.set_state(0, 0, q)
    for _ in range(20):
        H.step_level(0, dt=2.0)
    qg = H.get_state(0, 0)
    H.close()
    wet = q[0] > 1e-3
    assert np.abs((B + qg[3] + qg[0]) - (B + q[3] + q[0]))[wet].max() <= 1e-13 * 4000
    assert np.abs(qg[[1, 2, 4, 5]]).max() <= 1e-13 * 4000


def test_exchange_symmetry_on_the_gpu(mlswe_lib):
    """Transposed input (hu and hv exchanged) gives the transposed output to rounding."""
    n = 48
    q, B = I.gaussian_random_state(8, 2, n, n)

    def run(qq, BB):
        cfg = mlswe_lib.Config(M=2, dry_tol=1e-6, max_levels=1, unsplit=1)
        H = mlswe_lib.Hierarchy(cfg, [(0.0, 0.0, 1.0, 1.0, n, n)])
        H.set_bathymetry(0, BB)
        H.set_state(0, 0, qq)
        for _ in range(4):
            H.step_level(0, dt=0.3 / n / 4.0)
        out = H.get_state(0, 0)
        H.close()
        return out

    def swap(a):
        b = np.transpose(a, (0, 2, 1)).copy()
        b[[1, 2, 4, 5]] = b[[2, 1, 5, 4]]
        return b

    a = run(q, B)
    b = run(swap(q), B.T.copy())
    assert rel_err(swap(b), a).max() < 1e-12


def test_full_size_sampled(mlswe_lib):
    """2048^2 shelf workload, one unsplit step in the benchmark's launch configuration;
    sampled output cells checked against the oracle on their 9x9 input windows (a cell's
    update reads cells within two of it, corners included)."""
    w = I.scale(2048)
    q, B = w["q"], w["B"]
    n = 2048
    cfg = mlswe_lib.Config(M=2, dry_tol=1e-3, max_levels=1, unsplit=1)
    H = mlswe_lib.Hierarchy(cfg, [(0.0, 0.0, 1e5, 1e5, n, n)])
    H.set_bathymetry(0, B)
    H.set_state(0, 0, q)
    dt = 0.9 * w["dx"] / 205.0
    H.step_level(0, dt=dt)
    qg = H.get_state(0, 0)
    H.close()
    P = O.params(M=2, dry_tol=1e-3, unsplit=1)
    rs = np.random.default_rng(8)
    cells = [(int(rs.integers(4, n - 4)), int(rs.integers(4, n - 4))) for _ in range(48)]
    scale = np.maximum(state_scale(qg, 2), state_scale(q, 2))
    worst = np.zeros(6)
    for (j, i) in cells:
        sub = np.ascontiguousarray(q[:, j - 4:j + 5, i - 4:i + 5])
        subB = np.ascontiguousarray(B[j - 4:j + 5, i - 4:i + 5])
        O.step_patch(P, sub, subB, w["dx"], w["dy"], dt)
        ref = sub[:, 4, 4]
        err = np.abs(qg[:, j, i] - ref) / scale
        worst = np.maximum(worst, err)
        assert err.max() < TOL, (j, i, err)
    report("unsplit_scale_2048_sampled", worst)


def _amr_pair(pkg, levels, ratios, n, min_side, max_side, regrid, dynamic=0, Bf=None):
    nf = n * int(np.prod(ratios))
    if Bf is None:
        Bf = -np.ones((nf, nf))
    cfg = pkg.Config(M=2, dry_tol=1e-6, max_levels=levels, ratio=list(ratios) + [2] * 3, flag_tol=1e-3,
                     regrid_interval=regrid, n_buf=2, cluster_eff=0.7, min_side=min_side, max_side=max_side,
                     dynamic_rt=dynamic, unsplit=1)
    H = pkg.Hierarchy(cfg, [(0.0, 0.0, 1.0, 1.0, n, n)])
    H.set_bathymetry(0, Bf)
    A = OracleAMR(O.params(M=2, dry_tol=1e-6, unsplit=1), (0, 0, 1, 1), n, n, levels, list(ratios), Bf,
                  min_side=min_side, max_side=max_side, dynamic_rt=bool(dynamic))
    return H, A


def _compare(H, A):
    assert rel_err(H.get_state(0, 0), A.lev[0].q).max() < TOL
    for l in range(1, A.L):
        assert [tuple(b) for b in H.get_patches(0, l).tolist()] == [tuple(b) for b in A.lev[l].patches]
        m = A.lev[l].in_patch_mask()
        if m.any():
            assert rel_err(H.get_state(0, l)[:, m], A.lev[l].q[:, m]).max() < TOL


def test_amr_run_two_levels(mlswe_lib):
    """The small workload, ratio 2, regrid every 4 steps, 40 coarse steps: layouts identical,
    states within 1e-11, the clock equal; the composite mass of each layer constant."""
    w = I.small(50)
    H, A = _amr_pair(mlswe_lib, 2, (2,), 50, 16, 64, 4)
    H.set_state(0, 0, w["q"])
    A.set_state(0, w["q"])
    m0 = None
    for _ in range(10):
        H.advance(4)
        A.advance(4, regrid_interval=4)
        if m0 is None:
            m0 = A.mass()
        _compare(H, A)
    t, _ = H.get_time()
    assert abs(t[0] - A.t) <= 1e-12 * A.t
    assert np.all(np.abs(A.mass() - m0) <= 1e-13 * m0)
    H.close()


def test_amr_run_three_levels(mlswe_lib):
    w = I.small(40)
    H, A = _amr_pair(mlswe_lib, 3, (2, 2), 40, 8, 32, 3)
    H.set_state(0, 0, w["q"])
    A.set_state(0, w["q"])
    for _ in range(3):
        H.advance(3)
        A.advance(3, regrid_interval=3)
        _compare(H, A)
    assert len(A.lev[2].patches) > 0
    H.close()


def test_amr_dynamic_time_ratio(mlswe_lib):
    """Refined shallow half: the fine level takes fewer substeps than the ratio; the update
    kernel copies the state through the substeps the member skips."""
    n, r = 32, 4
    nf = n * r
    xf = (np.arange(nf) + 0.5) / nf
    Xf, _ = np.meshgrid(xf, xf)
    Bf = np.where(Xf < 0.5, -1.0, -0.05)
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x)
    B0 = O.bathy_average(Bf, r)
    q = np.zeros((6, n, n))
    q[3] = np.maximum(-0.02 - B0, 0.0)
    q[0] = 0.004 * np.exp(-((X - 0.75) ** 2 + (Y - 0.5) ** 2) / 0.004) - np.maximum(-0.02, B0)
    cfg = mlswe_lib.Config(M=2, rho=(1000.0, 1025.0), dry_tol=1e-6, max_levels=2, ratio=[r], flag_tol=2e-3,
                           regrid_interval=4, n_buf=2, cluster_eff=0.7, min_side=8, max_side=32, dynamic_rt=1,
                           unsplit=1)
    H = mlswe_lib.Hierarchy(cfg, [(0.0, 0.0, 1.0, 1.0, n, n)])
    H.set_bathymetry(0, Bf)
    H.set_state(0, 0, q)
    A = OracleAMR(O.params(M=2, rho=(1000.0, 1025.0), dry_tol=1e-6, unsplit=1), (0, 0, 1, 1), n, n, 2, [r], Bf,
                  flag_tol=2e-3, min_side=8, max_side=32, dynamic_rt=True)
    A.set_state(0, q)
    for _ in range(3):
        H.advance(4)
        A.advance(4, regrid_interval=4)
        _compare(H, A)
    assert H.get_stats()["level_steps"] == A.level_steps
    assert A.level_steps[1] < r * 12
    H.close()


RHO3 = (1000.0, 1020.0, 1030.0)


def _run_three(pkg, q, B, dx, dy, dts, order=2, dry_tol=1e-6):
    ny, nx = B.shape
    cfg = pkg.Config(M=3, rho=RHO3, order=order, dry_tol=dry_tol, max_levels=1, unsplit=1)
    H = pkg.Hierarchy(cfg, [(0.0, 0.0, nx * dx, ny * dy, nx, ny)])
    H.set_bathymetry(0, B)
    H.set_state(0, 0, q)
    P = O.params(M=3, rho=RHO3, dry_tol=dry_tol, order=order, unsplit=1)
    qo = q.copy()
    for dt in dts:
        H.step_level(0, dt=dt)
        qo, _, _ = O.step_walled(P, qo, B, dx, dy, dt)
    qg = H.get_state(0, 0)
    H.close()
    return qg, qo, P


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("shape", [(17, 23), (40, 130)])
def test_three_layer_random_wet_states(mlswe_lib, order, shape):
    """Three layers: the coupled transverse split reuses the normal solve's eigenvalues of the
    coupling matrix around the transverse mean velocity."""
    ny, nx = shape
    q, B = I.gaussian_random_state(51 + nx + ny, 3, nx, ny, depth=(0.5, 0.4, 0.6))
    dx, dy = 1.0 / nx, 1.3 / ny
    qg, qo, _ = _run_three(mlswe_lib, q, B, dx, dy, [0.25 * min(dx, dy) / 4.0] * 5, order=order)
    err = rel_err(qg, qo)
    assert err.max() < TOL, err


def test_three_layer_shore_and_rest(mlswe_lib):
    w = I.shore3(96, seed=3002)
    dts = [0.5 * w["dx"] / 210.0] * 20
    qg, qo, P = _run_three(mlswe_lib, w["q"], w["B"], w["dx"], w["dy"], dts, dry_tol=w["dry_tol"])
    err = state_err(qg, qo, 3)
    report("unsplit_three_layer_shore_96_20steps", err)
    assert err.max() < TOL, err
    n = 64
    B = I.shore_bathymetry(n, n)
    q = I.stacked_state(B, (np.zeros_like(B), -50.0 + 0.0 * B, -200.0 + 0.0 * B))
    cfg = mlswe_lib.Config(M=3, rho=RHO3, max_levels=1, unsplit=1)
    H = mlswe_lib.Hierarchy(cfg, [(0.0, 0.0, 1e5, 1e5, n, n)])
    H.set_bathymetry(0, B)
    H.set_state(0, 0, q)
    for _ in range(20):
        H.step_level(0, dt=2.0)
    qg = H.get_state(0, 0)
    H.close()
    assert np.abs(qg[[1, 2, 4, 5, 7, 8]]).max() <= 1e-13 * 4000


def test_options_the_unsplit_step_does_not_take(mlswe_lib):
    """The adjoint differentiates the split step only."""
    cfg = mlswe_lib.Config(M=2, dry_tol=1e-6, max_levels=1, order=1, unsplit=1)
    H = mlswe_lib.Hierarchy(cfg, [(0.0, 0.0, 1.0, 1.0, 40, 40)])
    q, B = I.gaussian_random_state(3, 2, 40, 40)
    H.set_bathymetry(0, B)
    H.set_state(0, 0, q)
    H.set_dt(0, 1e-4)
    with pytest.raises(mlswe_lib.MLSWEError) as e:
        H.adjoint_setup(10, 5, np.array([[3, 4]]), np.zeros((10, 1)))
    assert e.value.status == 1
    H.close()
