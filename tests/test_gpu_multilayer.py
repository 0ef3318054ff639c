"""Three layers on the GPU (the general M-layer coupled branch) against the oracle: random
wet states (both orders, odd shapes), a shore where the lower layers meet dry ground (the
per-layer branch and its walls), the lake at rest, the count of edges that lost
hyperbolicity, and a subcycled AMR run (refinement, coarsening and reflux with three layers).
Tolerance: 1e-11 relative per field; on the deep shore a momentum's scale is at least
h_max sqrt(g h_max) of its layer (state_scale), as in the two-layer tests."""
import numpy as np
import pytest

from paper_1803_01450_gb300 import inputs as I
from conftest import rel_err, report, state_err, state_scale

pytestmark = pytest.mark.gpu
TOL = 1e-11
RHO3 = (1000.0, 1020.0, 1030.0)


def _hier(pkg, nx, ny, dom, **kw):
    opts = dict(M=3, rho=RHO3, max_levels=1)
    opts.update(kw)
    return pkg.Hierarchy(pkg.Config(**opts), [(dom[0], dom[1], dom[2], dom[3], nx, ny)])


def _run_both(pkg, orc, q, B, dx, dy, dts, **kw):
    ny, nx = B.shape
    H = _hier(pkg, nx, ny, (0.0, 0.0, nx * dx, ny * dy), **kw)
    H.set_bathymetry(0, B)
    H.set_state(0, 0, q)
    P = orc.params(M=3, rho=RHO3, dry_tol=kw.get("dry_tol", 1e-3), order=kw.get("order", 2),
                   limiter=kw.get("limiter", 2), eigen=kw.get("eigen", 0))
    qo, lost_o = q.copy(), 0
    H.hyperbolicity_losses(reset=True)
    for dt in dts:
        H.step_level(0, dt=dt)
        qo, _, lost = orc.step_walled(P, qo, B, dx, dy, dt)
        lost_o += lost
    qg, lost_g = H.get_state(0, 0), H.hyperbolicity_losses()
    H.close()
    return qg, qo, lost_g, lost_o, P


@pytest.mark.parametrize("order,limiter", [(2, 2), (1, 0), (2, 1)])
@pytest.mark.parametrize("shape", [(17, 23), (64, 130)])
def test_three_layer_random_wet_states(mlswe_lib, orc, order, limiter, shape):
    ny, nx = shape
    q, B = I.gaussian_random_state(31 + nx + ny, 3, nx, ny, depth=(0.5, 0.4, 0.6))
    dx, dy = 1.0 / nx, 1.3 / ny
    dts = [0.2 * min(dx, dy) / 4.0] * 5
    qg, qo, lg, lo, _ = _run_both(mlswe_lib, orc, q, B, dx, dy, dts, order=order, limiter=limiter, dry_tol=1e-6)
    err = rel_err(qg, qo)
    assert err.max() < TOL, err
    assert lg == lo


def test_three_layer_guesses_only_variant(mlswe_lib, orc):
    q, B = I.gaussian_random_state(7, 3, 40, 33, depth=(0.5, 0.4, 0.6))
    dts = [0.2 / 40 / 4.0] * 4
    qg, qo, _, _, _ = _run_both(mlswe_lib, orc, q, B, 1.0 / 40, 1.0 / 33, dts, eigen=1, dry_tol=1e-6)
    assert rel_err(qg, qo).max() < TOL


def test_three_layer_hyperbolicity_loss(mlswe_lib, orc):
    """A band where the top two layers shear past each other beyond the pair's bound takes
    the guesses; the counts agree edge for edge and the states match."""
    nx, ny = 48, 40
    q, B = I.gaussian_random_state(41, 3, nx, ny, depth=(0.5, 0.4, 0.6))
    band = slice(15, 25)
    q[1, band] = 0.4 * q[0, band]
    q[4, band] = -0.4 * q[3, band]
    dts = [0.2 / 48 / 4.0] * 3
    qg, qo, lg, lo, _ = _run_both(mlswe_lib, orc, q, B, 1.0 / nx, 1.0 / ny, dts, dry_tol=1e-6)
    assert lo > 0 and lg == lo, (lg, lo)
    assert rel_err(qg, qo).max() < TOL


def test_three_layer_shore(mlswe_lib, orc):
    w = I.shore3(96, seed=3002)
    dts = [0.5 * w["dx"] / 210.0] * 20
    qg, qo, _, _, P = _run_both(mlswe_lib, orc, w["q"], w["B"], w["dx"], w["dy"], dts, dry_tol=w["dry_tol"])
    err = state_err(qg, qo, 3)
    report("three_layer_shore_96_20steps", err)
    assert err.max() < TOL, err


def test_three_layer_lake_at_rest(mlswe_lib):
    n = 64
    B = I.shore_bathymetry(n, n)
    q = I.stacked_state(B, (np.zeros_like(B), -50.0 + 0.0 * B, -200.0 + 0.0 * B))
    H = _hier(mlswe_lib, n, n, (0.0, 0.0, 1e5, 1e5))
    H.set_bathymetry(0, B)
    H.set_state(0, 0, q)
    for _ in range(20):
        H.step_level(0, dt=2.0)
    qg = H.get_state(0, 0)
    H.close()
    assert np.abs(qg[[1, 2, 4, 5, 7, 8]]).max() <= 1e-13 * 4000
    wet = q[0] > 1e-3
    eta1 = B + qg[6] + qg[3] + qg[0]
    assert np.abs(eta1 - (B + q[6] + q[3] + q[0]))[wet].max() <= 1e-13 * 4000


def test_three_layer_amr_run(mlswe_lib):
    """20 coarse steps of a two-level (ratio 2) three-layer run with regrids every 4 steps:
    patch layouts identical, states within 1e-11, mass per layer equal to the oracle's."""
    from oracle.amr import OracleAMR
    import oracle as O
    n, r = 50, 2
    x = (np.arange(n * r) + 0.5) / (n * r)
    Xf, Yf = np.meshgrid(x, x)
    Bf = -1.5 + 0.2 * Xf
    cfg = mlswe_lib.Config(M=3, rho=RHO3, dry_tol=1e-6, max_levels=2, ratio=[r], flag_tol=1e-3, regrid_interval=4,
                           n_buf=2, cluster_eff=0.7, min_side=16, max_side=64)
    H = mlswe_lib.Hierarchy(cfg, [(0.0, 0.0, 1.0, 1.0, n, n)])
    H.set_bathymetry(0, Bf)
    B0 = H.get_bathymetry(0, 0)
    xc = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(xc, xc)
    eta1 = 0.02 * np.exp(-((X - 0.3) ** 2 + (Y - 0.5) ** 2) / 0.005)
    q0 = I.stacked_state(B0, (eta1, -0.4 + 0.0 * X, -0.8 + 0.0 * X))
    H.set_state(0, 0, q0)
    A = OracleAMR(O.params(M=3, rho=RHO3, dry_tol=1e-6), (0, 0, 1, 1), n, n, 2, [r], Bf, min_side=16, max_side=64)
    A.set_state(0, q0)
    for _ in range(5):
        H.advance(4)
        A.advance(4, regrid_interval=4)
        assert [tuple(b) for b in H.get_patches(0, 1).tolist()] == [tuple(b) for b in A.lev[1].patches]
    assert rel_err(H.get_state(0, 0), A.lev[0].q).max() < TOL
    m = A.lev[1].in_patch_mask()
    assert rel_err(H.get_state(0, 1)[:, m], A.lev[1].q[:, m]).max() < TOL
    H.close()
