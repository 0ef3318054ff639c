"""GPU parity of the fixed-grid (single level) step against the FP64 oracle.

Tolerance: 1e-11 relative per field (max abs difference over the field divided by the
field's max magnitude), the bound stated for the state after N steps. The CUDA path
reaches the same formulas through reciprocals, a closed-form Vandermonde solve of the
wave strengths and fused multiply-adds, so the two agree to rounding, not bit for bit.
"""
import numpy as np
import pytest

from paper_1803_01450_gb300 import inputs as I
from conftest import rel_err, report, state_err, state_scale

pytestmark = pytest.mark.gpu
TOL = 1e-11


def _hier(pkg, M, nx, ny, dom, order=2, limiter=2, dry_tol=1e-3, eigen=0):
    cfg = pkg.Config(M=M, order=order, limiter=limiter, dry_tol=dry_tol, eigen=eigen, max_levels=1)
    return pkg.Hierarchy(cfg, [(dom[0], dom[1], dom[2], dom[3], nx, ny)])


def _run_both(pkg, orc, q, B, dx, dy, dts, M=2, order=2, limiter=2, dry_tol=1e-3, eigen=0):
    ny, nx = B.shape
    H = _hier(pkg, M, nx, ny, (0.0, 0.0, nx * dx, ny * dy), order, limiter, dry_tol, eigen)
    H.set_bathymetry(0, B)
    H.set_state(0, 0, q)
    P = orc.params(M=M, dry_tol=dry_tol, order=order, limiter=limiter, eigen=eigen)
    qo = q.copy()
    for dt in dts:
        H.step_level(0, dt=dt)
        qo, _, _ = orc.step_walled(P, qo, B, dx, dy, dt)
    qg = H.get_state(0, 0)
    H.close()
    return qg, qo


def test_small_config_100_steps(mlswe_lib, orc):
    w = I.small(50)
    dts = [0.9 * w["dx"] / 3.2] * 100
    qg, qo = _run_both(mlswe_lib, orc, w["q"], w["B"], w["dx"], w["dy"], dts, dry_tol=w["dry_tol"])
    err = rel_err(qg, qo)
    report("small_50_100steps", err)
    assert err.max() < TOL, err


@pytest.mark.parametrize("M,order,limiter", [(2, 2, 2), (2, 1, 0), (2, 2, 1), (1, 2, 2), (1, 1, 0)])
@pytest.mark.parametrize("shape", [(17, 23), (64, 130), (5, 300)])
def test_random_wet_states(mlswe_lib, orc, M, order, limiter, shape):
    ny, nx = shape
    q, B = I.gaussian_random_state(11 + nx + 7 * ny + M, M, nx, ny)
    dx, dy = 1.0 / nx, 1.3 / ny
    dts = [0.2 * min(dx, dy) / 4.0] * 5
    qg, qo = _run_both(mlswe_lib, orc, q, B, dx, dy, dts, M=M, order=order, limiter=limiter, dry_tol=1e-6)
    err = rel_err(qg, qo)
    report(f"random_M{M}_o{order}_l{limiter}_{ny}x{nx}", err)
    assert err.max() < TOL, err


def test_eigen_guess_only_variant(mlswe_lib, orc):
    q, B = I.gaussian_random_state(5, 2, 40, 33)
    dts = [0.2 / 40 / 4.0] * 4
    qg, qo = _run_both(mlswe_lib, orc, q, B, 1 / 40, 1 / 33, dts, eigen=1, dry_tol=1e-6)
    assert rel_err(qg, qo).max() < TOL


def test_shore_wet_dry(mlswe_lib, orc):
    """Shelf + shore with both layers meeting dry land, 20 steps. Deep water (B down to
    -4000 m) makes the momentum of the near-rest region rounding noise of the well-balanced
    eta - B reconstruction; momenta are measured against the physical scale
    h_max sqrt(g h_max) of their layer (state_scale)."""
    w = I.shore(96, seed=3001)
    dts = [0.5 * w["dx"] / 210.0] * 20
    qg, qo = _run_both(mlswe_lib, orc, w["q"], w["B"], w["dx"], w["dy"], dts, dry_tol=w["dry_tol"])
    err = state_err(qg, qo, 2)
    report("shore_96_20steps", err)
    assert err.max() < TOL, err


def test_lake_at_rest_gpu(mlswe_lib):
    n = 64
    B = I.shore_bathymetry(n, n)
    q = I.layered_state(B, np.zeros_like(B), -200.0 * np.ones_like(B))
    H = _hier(mlswe_lib, 2, n, n, (0.0, 0.0, 1e5, 1e5))
    H.set_bathymetry(0, B)
    H.set_state(0, 0, q)
    for _ in range(20):
        H.step_level(0, dt=2.0)
    qg = H.get_state(0, 0)
    H.close()
    eta1 = B + qg[3] + qg[0]
    wet = q[0] > 1e-3
    assert np.abs(eta1 - (B + q[3] + q[0]))[wet].max() <= 1e-13 * 4000
    assert np.abs(qg[[1, 2, 4, 5]]).max() <= 1e-13 * 4000


def test_cfl_report(mlswe_lib, orc):
    w = I.small(50)
    H = _hier(mlswe_lib, 2, 50, 50, (0.0, 0.0, 1.0, 1.0), dry_tol=w["dry_tol"])
    H.set_bathymetry(0, w["B"])
    H.set_state(0, 0, w["q"])
    dt = 0.004
    cfl = H.step_level(0, dt=dt, want_cfl=True)
    H.close()
    P = orc.params(M=2, dry_tol=w["dry_tol"])
    _, smax, _ = orc.step_walled(P, w["q"], w["B"], w["dx"], w["dy"], dt)
    ref = dt * max(smax[0] / w["dx"], smax[1] / w["dy"])
    assert abs(cfl[0] - ref) <= 1e-12 * ref


def test_full_size_sampled(mlswe_lib, orc):
    """2048^2 shelf workload, one step in the benchmark's launch configuration; sampled
    output cells checked against the oracle on their 9x9 input windows."""
    w = I.scale(2048)
    q, B = w["q"], w["B"]
    n = 2048
    H = _hier(mlswe_lib, 2, n, n, (0.0, 0.0, 1e5, 1e5))
    H.set_bathymetry(0, B)
    H.set_state(0, 0, q)
    dt = 0.9 * w["dx"] / 205.0
    H.step_level(0, dt=dt)
    qg = H.get_state(0, 0)
    H.close()
    P = orc.params(M=2, dry_tol=1e-3)
    rs = np.random.default_rng(7)
    cells = [(int(rs.integers(4, n - 4)), int(rs.integers(4, n - 4))) for _ in range(48)]
    # per-field scale of the whole state before and after the step (momenta start at zero,
    # so they take the physical scale h_max sqrt(g h_max) of their layer, state_scale)
    scale = np.maximum(state_scale(qg, 2), state_scale(q, 2))
    worst = np.zeros(6)
    for (j, i) in cells:
        sub = np.ascontiguousarray(q[:, j - 4:j + 5, i - 4:i + 5])
        subB = np.ascontiguousarray(B[j - 4:j + 5, i - 4:i + 5])
        orc.step_patch(P, sub, subB, w["dx"], w["dy"], dt)
        ref = sub[:, 4, 4]
        err = np.abs(qg[:, j, i] - ref) / scale
        worst = np.maximum(worst, err)
        assert err.max() < TOL, (j, i, err)
    report("scale_2048_sampled", worst)


def test_hyperbolicity_loss_branch(mlswe_lib, orc):
    """A band where the layers shear past each other ((u1 - u2)^2 = 1 above (1 - r) g (h1 + h2)
    = 0.36) takes the guesses-only branch at its edges: the state matches the oracle and the
    count of such edges equals the oracle's, each edge counted once."""
    nx, ny = 48, 40
    q, B = I.gaussian_random_state(21, 2, nx, ny)
    band = slice(15, 25)
    q[1, band] = 0.5 * q[0, band]
    q[4, band] = -0.5 * q[3, band]
    dx, dy = 1.0 / nx, 1.0 / ny
    dts = [0.2 * min(dx, dy) / 4.0] * 3
    H = _hier(mlswe_lib, 2, nx, ny, (0.0, 0.0, 1.0, 1.0), dry_tol=1e-6)
    H.set_bathymetry(0, B)
    H.set_state(0, 0, q)
    H.hyperbolicity_losses(reset=True)
    P = orc.params(M=2, dry_tol=1e-6)
    qo, lost_o = q.copy(), 0
    for dt in dts:
        H.step_level(0, dt=dt)
        qo, _, lost = orc.step_walled(P, qo, B, dx, dy, dt)
        lost_o += lost
    lost_g = H.hyperbolicity_losses()
    assert lost_o > 0 and lost_g == lost_o, (lost_g, lost_o)
    err = rel_err(H.get_state(0, 0), qo)
    assert err.max() < TOL, err
    # no shear, no loss
    H.set_state(0, 0, I.gaussian_random_state(22, 2, nx, ny)[0])
    H.step_level(0, dt=dts[0])
    assert H.hyperbolicity_losses() == 0
    H.close()
