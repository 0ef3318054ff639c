"""FP64 CPU oracle for the multilayer shallow-water AMR hot path.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The CUDA library never
imports, links or calls it, and it shares no code with the library.

The numerical core is ``mlswe_oracle.cpp`` (plain loops, ``-ffp-contract=off``);
this module only loads it through ctypes and offers numpy-shaped wrappers. The
AMR driver built on top of these primitives is in :mod:`oracle.amr`, the
patch clustering in :mod:`oracle.cluster`.

Paper: arXiv:1803.01450 (Schwarzschild & Mandli). Each wrapper names the
passage of the paper it follows; the solver step, which the paper does not
write out, follows the reading stated in ``mlswe_oracle.cpp``.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mlswe_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_TIMING_LIB_PATH = os.path.join(_BUILD, "liboracle_timing.so")
_lib = None
_use_timing = False

NG = 2


def _compile(out, flags):
    cmd = ["g++", *flags, "-std=c++17", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-o", out + ".tmp",
           _SRC]
    subprocess.check_call(cmd)
    os.replace(out + ".tmp", out)


def build(force: bool = False) -> str:
    """Compile the oracle shared library (g++, OpenMP, no FP contraction): the parity build
    (-O2) and the build the CPU baseline is timed with (-O3, and on Arm hosts scheduled for
    the Grace CPU's Neoverse V2 cores; same arithmetic: no contraction, no reassociation)."""
    import concurrent.futures as cf
    os.makedirs(_BUILD, exist_ok=True)
    stale = lambda p: force or not os.path.exists(p) or os.path.getmtime(p) < os.path.getmtime(_SRC)

    def timing():
        # scheduling tuned for the Grace CPU's Neoverse V2 cores, no instruction-set extension
        # (SVE instructions stopped a run with SIGILL on a host that does not enable them)
        tuned = ["-O3", "-mtune=neoverse-v2"] if platform.machine() in ("aarch64", "arm64") else ["-O3"]
        try:
            _compile(_TIMING_LIB_PATH, tuned)
        except subprocess.CalledProcessError:
            _compile(_TIMING_LIB_PATH, ["-O3"])

    jobs = ([lambda: _compile(_LIB_PATH, ["-O2"])] if stale(_LIB_PATH) else []) + \
        ([timing] if stale(_TIMING_LIB_PATH) else [])
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        for f in [ex.submit(j) for j in jobs]:
            f.result()
    return _TIMING_LIB_PATH if _use_timing else _LIB_PATH


def use_timing_build() -> None:
    """Load the timing build instead of the parity build (before the first oracle call)."""
    global _use_timing
    if _lib is not None and not _use_timing:
        raise RuntimeError("oracle: the parity build is already loaded")
    _use_timing = True


def threads() -> int:
    """OpenMP threads of the oracle's parallel loops."""
    return int(lib().or_threads())


MAXM = 4  # layers the oracle supports (MAXM in mlswe_oracle.cpp)


class Params(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("g", ctypes.c_double), ("r", ctypes.c_double),
                ("dry_tol", ctypes.c_double), ("order", ctypes.c_int), ("limiter", ctypes.c_int),
                ("eigen", ctypes.c_int), ("rho", ctypes.c_double * MAXM), ("unsplit", ctypes.c_int)]


def params(M=2, g=9.81, rho=None, dry_tol=1e-3, order=2, limiter=2, eigen=0, unsplit=0) -> Params:
    """rho: layer densities, top (lightest) first; default 1000, 1025 for two layers and
    1000, 1020, 1030, 1040 (first M) otherwise. unsplit: 1 for the unsplit step with
    transverse Riemann solves (wave propagation in corner-transport form), 0 for
    dimensional splitting."""
    if rho is None:
        rho = (1000.0, 1025.0) if M == 2 else (1000.0, 1020.0, 1030.0, 1040.0)[:M]
    r = rho[0] / rho[1] if M == 2 else 1.0
    rr = (ctypes.c_double * MAXM)(*(list(rho[:M]) + [0.0] * (MAXM - min(M, len(rho)))))
    return Params(M, g, r, dry_tol, order, limiter, eigen, rr, unsplit)


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_pp = ctypes.POINTER(Params)


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        L.or_riemann.argtypes = [_pp, _dp, _dp, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp, _dp, _ip]
        L.or_riemann_general.argtypes = [_pp, _dp, _dp, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp, _dp, _ip]
        L.or_transverse.argtypes = [_pp, _dp, _dp, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp, ctypes.c_int]
        L.or_eigen.argtypes = [_pp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp, _ip]
        L.or_sweep_line.argtypes = [_pp, ctypes.c_int, _dp, _dp, ctypes.c_double, _dp, _dp]
        L.or_sweep_line.restype = ctypes.c_double
        L.or_fill_walls.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_int]
        L.or_step_patch.argtypes = [_pp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, _dp, _dp, _dp, _dp, _dp]
        L.or_step_patch.restype = ctypes.c_int
        L.or_step_walled.argtypes = [_pp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, _dp, _dp, _dp]
        L.or_step_walled.restype = ctypes.c_int
        L.or_interp_fine.argtypes = [_pp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp]
        L.or_average_coarse.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp]
        L.or_flags.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _u8p, ctypes.c_double,
                               ctypes.c_double, ctypes.c_double, ctypes.c_double, _u8p]
        L.or_bathy_average.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp]
        L.or_count_sweep.argtypes = [_pp, ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.POINTER(ctypes.c_longlong)]
        L.or_count_unsplit.argtypes = [_pp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, _dp, _dp, ctypes.POINTER(ctypes.c_longlong)]
        L.or_threads.restype = ctypes.c_int
        L.or_adjoint_step.argtypes = [_pp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, _dp, _dp, _dp, _dp]
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _c(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


# --------------------------------------------------------------------------- edge level
def riemann(P: Params, qL, qR, BL, BR, general=False):
    """Waves, speeds and fluctuations at one edge (normal direction first in each layer).

    Returns (Z[3W][3W], s[3W], amdq[3W], apdq[3W], info) with W = max(M, 2): waves and
    fields beyond 3M are zero; info = (wall side of each of the first W layers,
    hyperbolicity-loss flag). general: take the general M-layer coupled branch also for
    M = 2."""
    F, W = 3 * MAXM, max(P.M, 2)
    qL = _c(np.pad(np.asarray(qL, float), (0, F - len(qL))))
    qR = _c(np.pad(np.asarray(qR, float), (0, F - len(qR))))
    Z = np.zeros((F, F)); s = np.zeros(F); am = np.zeros(F); ap = np.zeros(F)
    info = np.zeros(MAXM + 1, dtype=np.int32)
    fn = lib().or_riemann_general if general else lib().or_riemann
    fn(ctypes.byref(P), _d(qL), _d(qR), float(BL), float(BR), _d(Z), _d(s), _d(am), _d(ap),
       info.ctypes.data_as(_ip))
    n = 3 * W
    return Z[:n, :n].copy(), s[:n].copy(), am[:n].copy(), ap[:n].copy(), np.concatenate([info[:W], info[MAXM:]])


def transverse(P: Params, qL, qR, BL, BR, dq, general=False):
    """Transverse split of the fluctuation dq (3M, normal-frame order (h, hn, ht) per layer)
    at the edge (qL, qR, BL, BR): returns (bp, bm), the parts carried towards +t and -t."""
    F = 3 * MAXM
    pad = lambda v: _c(np.pad(np.asarray(v, float), (0, F - len(v))))
    bp = np.zeros(F); bm = np.zeros(F)
    lib().or_transverse(ctypes.byref(P), _d(pad(qL)), _d(pad(qR)), float(BL), float(BR), _d(pad(dq)), _d(bp),
                        _d(bm), int(general))
    n = 3 * P.M
    return bp[:n].copy(), bm[:n].copy()


def eigen(P: Params, u1, u2, hb1, hb2):
    lam = np.zeros(4)
    lost = ctypes.c_int(0)
    lib().or_eigen(ctypes.byref(P), float(u1), float(u2), float(hb1), float(hb2), _d(lam), ctypes.byref(lost))
    return lam, lost.value


def sweep_line(P: Params, line, Bline, nu):
    """1-D sweep of n cells; line is [n+4][3M] (two ghosts per end), Bline [n+4]."""
    line = _c(line); Bline = _c(Bline)
    n = line.shape[0] - 4
    F = 3 * P.M
    out = np.zeros((n, F))
    mf = np.zeros((n + 1, P.M))
    s = lib().or_sweep_line(ctypes.byref(P), n, _d(line), _d(Bline), float(nu), _d(out), _d(mf))
    return out, s, mf


def count_sweep(P: Params, line, Bline, nu):
    """(additions, multiplications, divisions, square roots) of one 1-D sweep of the method
    over a line of n cells (two ghosts per end), counted by the oracle's counting scalar."""
    line = _c(line); Bline = _c(Bline)
    out = (ctypes.c_longlong * 4)()
    lib().or_count_sweep(ctypes.byref(P), line.shape[0] - 4, _d(line), _d(Bline), float(nu), out)
    return tuple(int(v) for v in out)


def flops_per_cell_update(P: Params, q, B, dx, dy, dt, rows, cols):
    """FP64 operations of the method per cell update (x sweep + y sweep, one flop per +, -,
    *, / and sqrt), averaged over the given interior rows (x sweep) and columns (y sweep)
    of a dense state q [3M][ny][nx]; the halo edges of a line are charged to the line."""
    F = 3 * P.M
    ny, nx = B.shape
    tot, cells = 0, 0
    for j in rows:
        line = np.zeros((nx + 4, F))
        line[2:-2] = q[:, j, :].T
        line[:2] = line[2:4][::-1]; line[-2:] = line[-4:-2][::-1]
        for m in range(P.M):
            line[:2, 3 * m + 1] *= -1; line[-2:, 3 * m + 1] *= -1
        Bl = np.concatenate([B[j, :2][::-1], B[j], B[j, -2:][::-1]])
        tot += sum(count_sweep(P, line, Bl, dt / dx)); cells += nx
    for i in cols:
        line = np.zeros((ny + 4, F))
        for m in range(P.M):
            line[2:-2, 3 * m] = q[3 * m, :, i]
            line[2:-2, 3 * m + 1] = q[3 * m + 2, :, i]
            line[2:-2, 3 * m + 2] = q[3 * m + 1, :, i]
        line[:2] = line[2:4][::-1]; line[-2:] = line[-4:-2][::-1]
        for m in range(P.M):
            line[:2, 3 * m + 1] *= -1; line[-2:, 3 * m + 1] *= -1
        Bl = np.concatenate([B[:2, i][::-1], B[:, i], B[-2:, i][::-1]])
        tot += sum(count_sweep(P, line, Bl, dt / dy)); cells += ny
    # one x sweep and one y sweep per cell update
    return 2.0 * tot / cells


def flops_per_cell_update_unsplit(P: Params, q, B, dx, dy, dt, windows):
    """FP64 operations of the unsplit step per cell update, by phase, counted on n x n
    windows (i0, j0, n) of a dense state q [3M][ny][nx] with their two-cell rings taken from
    q (windows away from the walls). The edge passes solve n + 2 lines of n cells (one ghost
    line per side); their per-line cost is charged to the n interior lines only, so 'x' and
    'y' are the work of the edges of one cell, 'update' that of the transverse correction
    fluxes and the cell update. Returns a dict x, y, update, total."""
    tot = np.zeros(4)
    cells = 0
    for (i0, j0, n) in windows:
        qp = _c(q[:, j0 - NG:j0 + n + NG, i0 - NG:i0 + n + NG])
        Bp = _c(B[j0 - NG:j0 + n + NG, i0 - NG:i0 + n + NG])
        out = (ctypes.c_longlong * 16)()
        lib().or_count_unsplit(ctypes.byref(P), n, n, float(dx), float(dy), float(dt), _d(qp), _d(Bp), out)
        ph = np.array(out, dtype=float).reshape(4, 4).sum(axis=1)
        tot += np.array([ph[0] / (n + 2) * n, ph[1] / (n + 2) * n, ph[2], ph[3]])
        cells += n * n
    x, y, upd = tot[0] / cells, tot[1] / cells, (tot[2] + tot[3]) / cells
    return {"x": x, "y": y, "update": upd, "total": x + y + upd}


# --------------------------------------------------------------------------- grid level
def pad(q, B=None):
    """Dense [F][ny][nx] (and [ny][nx]) -> patch arrays with a zero ghost ring of 2."""
    qp = np.pad(np.asarray(q, float), ((0, 0), (NG, NG), (NG, NG)))
    if B is None:
        return _c(qp)
    return _c(qp), _c(np.pad(np.asarray(B, float), ((NG, NG), (NG, NG))))


def fill_walls(M, qp, Bp=None, sides=15):
    F, H, W = qp.shape
    assert F == 3 * M and qp.flags.c_contiguous
    lib().or_fill_walls(M, W - 2 * NG, H - 2 * NG, _d(qp), _d(Bp) if Bp is not None else None, sides)


def step_patch(P: Params, qp, Bp, dx, dy, dt, want_flux=False):
    """One step (split, or unsplit with P.unsplit) on a patch array with its ghost ring
    already filled (in place).

    Returns (smax[2], lost, fx, fy) with fx [M][ny][nx+1], fy [M][ny+1][nx] mass fluxes."""
    assert qp.flags.c_contiguous and Bp.flags.c_contiguous
    F, H, W = qp.shape
    nx, ny = W - 2 * NG, H - 2 * NG
    smax = np.zeros(2)
    fx = np.zeros((P.M, ny, nx + 1)) if want_flux else None
    fy = np.zeros((P.M, ny + 1, nx)) if want_flux else None
    lost = lib().or_step_patch(ctypes.byref(P), nx, ny, float(dx), float(dy), float(dt), _d(qp), _d(Bp),
                               _d(smax), _d(fx) if want_flux else None, _d(fy) if want_flux else None)
    return smax, lost, fx, fy


def step_walled(P: Params, q, B, dx, dy, dt):
    """One step of a dense walled grid q [3M][ny][nx]; returns (q_new, smax[2], lost)."""
    qp, Bp = pad(q, B)
    fill_walls(P.M, qp, Bp)
    smax, lost, _, _ = step_patch(P, qp, Bp, dx, dy, dt)
    return qp[:, NG:-NG, NG:-NG].copy(), smax, lost


def interp_fine(P: Params, r, qc_padded, Bc_padded, box, Bf):
    """Refinement of the coarse cells box = (ci0, cj0, ci1, cj1) (Sec. 2.1).

    qc_padded: coarse patch array with a valid ghost ring. Bf: fine bathymetry of the box."""
    ci0, cj0, ci1, cj1 = box
    F, H, W = qc_padded.shape
    nxc, nyc = W - 2 * NG, H - 2 * NG
    Bf = _c(Bf)
    assert Bf.shape == ((cj1 - cj0) * r, (ci1 - ci0) * r)
    out = np.zeros((F, (cj1 - cj0) * r, (ci1 - ci0) * r))
    lib().or_interp_fine(ctypes.byref(P), int(r), nxc, nyc, _d(_c(qc_padded)), _d(_c(Bc_padded)),
                         ci0, cj0, ci1, cj1, _d(Bf), _d(out))
    return out


def average_coarse(qf, r):
    """Coarsening, Sec. 2.2 Eq. (11): [nf][nyf][nxf] -> [nf][nyf/r][nxf/r]."""
    qf = _c(qf)
    squeeze = qf.ndim == 2
    if squeeze:
        qf = qf[None]
    nf, nyf, nxf = qf.shape
    assert nyf % r == 0 and nxf % r == 0
    out = np.zeros((nf, nyf // r, nxf // r))
    lib().or_average_coarse(nf, int(r), nxf, nyf, _d(qf), _d(out))
    return out[0] if squeeze else out


def bathy_average(Bf, r):
    return average_coarse(Bf, r)


def flags(M, q, B, avail, dry_tol, dx, dy, tol):
    """Gradient flags of eta_1 (dense level arrays); inv_dx etc. computed here once."""
    q = _c(q); B = _c(B); avail = _c(avail, np.uint8)
    F, ny, nx = q.shape
    out = np.zeros((ny, nx), dtype=np.uint8)
    lib().or_flags(M, nx, ny, _d(q), _d(B), avail.ctypes.data_as(_u8p), float(dry_tol), 1.0 / dx, 1.0 / dy,
                   float(tol) * float(tol), out.ctypes.data_as(_u8p))
    return out


def adjoint_step(P: Params, qn, B, dx, dy, dt, lam):
    """Transpose of the first-order step Jacobian applied to lam; returns (lam_n, gB)."""
    qn = _c(qn); B = _c(B); lam = _c(lam).copy()
    F, ny, nx = qn.shape
    gB = np.zeros((ny, nx))
    lib().or_adjoint_step(ctypes.byref(P), nx, ny, float(dx), float(dy), float(dt), _d(qn), _d(B), _d(lam), _d(gB))
    return lam, gB
