"""The three- and four-layer 2048^2 shelf workloads (the bench's three_layers and four_layers
figures) at full size: one step in the benchmark's launch configuration (autotuned tiles, one
CTA per SM), and sampled output cells checked against the oracle on their 9 x 9 input windows
(the split second-order step reaches four cells), within 1e-11 of each field's scale
(state_scale); the three-layer workload also through the unsplit step. The samples include
shelf cells where the lower layers end (the per-layer branch of the edge solve) besides the
deep water of the coupled M-layer branch."""
import numpy as np
import pytest

from paper_1803_01450_gb300 import inputs as I
from conftest import report, state_scale

pytestmark = pytest.mark.gpu
TOL = 1e-11
RHO = {3: (1000.0, 1020.0, 1030.0), 4: (1000.0, 1020.0, 1030.0, 1040.0)}


@pytest.mark.parametrize("M", [3, 4])
def test_multilayer_full_size_sampled(mlswe_lib, orc, M):
    pkg = mlswe_lib
    n = 2048
    w = I.scale3(n, seed=1000) if M == 3 else I.scale4(n, seed=1000)
    q, B = w["q"], w["B"]
    cfg = pkg.Config(M=M, rho=RHO[M], dry_tol=w["dry_tol"], order=2, limiter=2, max_levels=1)
    H = pkg.Hierarchy(cfg, [(0.0, 0.0, 1e5, 1e5, n, n)])
    H.set_bathymetry(0, B)
    H.set_state(0, 0, q)
    H.autotune(0, iters=1)
    dt = 0.9 * w["dx"] / 205.0
    H.step_level(0, dt=dt)
    qg = H.get_state(0, 0)
    H.close()
    P = orc.params(M=M, rho=RHO[M], dry_tol=w["dry_tol"], order=2, limiter=2)
    rs = np.random.default_rng(11 + M)
    cells = [(int(rs.integers(4, n - 4)), int(rs.integers(4, n - 4))) for _ in range(40)]
    # and eight on the shelf, where the lower layers end (x beyond about 62 km)
    cells += [(int(rs.integers(4, n - 4)), int(rs.integers(int(0.62 * n), n - 4))) for _ in range(8)]
    shallow = sum(1 for (j, i) in cells if q[3 * (M - 1), j, i] <= w["dry_tol"])
    assert shallow > 0
    scale = np.maximum(state_scale(qg, M), state_scale(q, M))
    worst = np.zeros(3 * M)
    for (j, i) in cells:
        sub = np.ascontiguousarray(q[:, j - 4:j + 5, i - 4:i + 5])
        subB = np.ascontiguousarray(B[j - 4:j + 5, i - 4:i + 5])
        orc.step_patch(P, sub, subB, w["dx"], w["dy"], dt)
        err = np.abs(qg[:, j, i] - sub[:, 4, 4]) / scale
        worst = np.maximum(worst, err)
        assert err.max() < TOL, (j, i, err)
    report(f"scale_2048_M{M}_sampled", worst)


def test_three_layer_unsplit_full_size_sampled(mlswe_lib, orc):
    """The same three-layer workload through the unsplit step (transverse Riemann solves),
    sampled the same way (a cell's unsplit update reads cells within two of it, corners
    included)."""
    pkg = mlswe_lib
    n, M = 2048, 3
    w = I.scale3(n, seed=1000)
    q, B = w["q"], w["B"]
    cfg = pkg.Config(M=M, rho=RHO[M], dry_tol=w["dry_tol"], order=2, limiter=2, max_levels=1, unsplit=1)
    H = pkg.Hierarchy(cfg, [(0.0, 0.0, 1e5, 1e5, n, n)])
    H.set_bathymetry(0, B)
    H.set_state(0, 0, q)
    dt = 0.9 * w["dx"] / 205.0
    H.step_level(0, dt=dt)
    qg = H.get_state(0, 0)
    H.close()
    P = orc.params(M=M, rho=RHO[M], dry_tol=w["dry_tol"], order=2, limiter=2, unsplit=1)
    rs = np.random.default_rng(23)
    cells = [(int(rs.integers(4, n - 4)), int(rs.integers(4, n - 4))) for _ in range(32)]
    cells += [(int(rs.integers(4, n - 4)), int(rs.integers(int(0.62 * n), n - 4))) for _ in range(8)]
    scale = np.maximum(state_scale(qg, M), state_scale(q, M))
    worst = np.zeros(3 * M)
    for (j, i) in cells:
        sub = np.ascontiguousarray(q[:, j - 4:j + 5, i - 4:i + 5])
        subB = np.ascontiguousarray(B[j - 4:j + 5, i - 4:i + 5])
        orc.step_patch(P, sub, subB, w["dx"], w["dy"], dt)
        err = np.abs(qg[:, j, i] - sub[:, 4, 4]) / scale
        worst = np.maximum(worst, err)
        assert err.max() < TOL, (j, i, err)
    report("unsplit_scale_2048_M3_sampled", worst)
