"""GB300-native multilayer shallow-water AMR (arXiv:1803.01450), Python binding.

This module only marshals arguments to the C ABI declared in ``include/mlswe.h``
(``lib/libmlswe.so``, built in tree by :func:`build`). Every step of the hot
path runs in the library's CUDA kernels; there is no CPU fallback, and every
entry point raises if the library or a CUDA device is missing.

PyTorch provides device memory (through the allocator callback of the C ABI)
and the CUDA stream; nothing else.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build_mod

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libmlswe.so")

MLSWE_OK = 0
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ECFL", 5: "ENEGDEPTH", 6: "ENESTING",
                7: "ETIMEOUT", 8: "EHYPERB", 9: "EMISSING"}


class MLSWEError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"mlswe {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class _Config(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("rho", ctypes.c_double * 4), ("g", ctypes.c_double),
                ("dry_tol", ctypes.c_double), ("cfl_desired", ctypes.c_double), ("cfl_max", ctypes.c_double),
                ("order", ctypes.c_int), ("limiter", ctypes.c_int), ("eigen", ctypes.c_int),
                ("max_levels", ctypes.c_int), ("ratio", ctypes.c_int * 4), ("flag_tol", ctypes.c_double),
                ("regrid_interval", ctypes.c_int), ("n_buf", ctypes.c_int), ("cluster_eff", ctypes.c_double),
                ("min_side", ctypes.c_int), ("max_side", ctypes.c_int), ("dynamic_rt", ctypes.c_int),
                ("unsplit", ctypes.c_int)]


class _Domain(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_double), ("y0", ctypes.c_double), ("x1", ctypes.c_double),
                ("y1", ctypes.c_double), ("nx0", ctypes.c_int), ("ny0", ctypes.c_int)]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class _Allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("ctx", ctypes.c_void_p)]


@dataclasses.dataclass
class Config:
    """Mirror of ``mlswe_config`` (see include/mlswe.h)."""
    M: int = 2
    rho: Sequence[float] = (1000.0, 1025.0)
    g: float = 9.81
    dry_tol: float = 1e-3
    cfl_desired: float = 0.9
    cfl_max: float = 1.0
    order: int = 2
    limiter: int = 2
    eigen: int = 0
    max_levels: int = 1
    ratio: Sequence[int] = (4, 4, 4)
    flag_tol: float = 1e-3
    regrid_interval: int = 4
    n_buf: int = 2
    cluster_eff: float = 0.7
    min_side: int = 16
    max_side: int = 64
    dynamic_rt: int = 0
    unsplit: int = 0

    def to_c(self) -> _Config:
        c = _Config()
        c.M = self.M
        rho = list(self.rho) + [0.0] * (4 - len(self.rho))
        for k in range(4):
            c.rho[k] = rho[k]
        c.g = self.g; c.dry_tol = self.dry_tol; c.cfl_desired = self.cfl_desired; c.cfl_max = self.cfl_max
        c.order = self.order; c.limiter = self.limiter; c.eigen = self.eigen; c.max_levels = self.max_levels
        rat = list(self.ratio) + [2] * (4 - len(self.ratio))
        for k in range(4):
            c.ratio[k] = rat[k]
        c.flag_tol = self.flag_tol; c.regrid_interval = self.regrid_interval; c.n_buf = self.n_buf
        c.cluster_eff = self.cluster_eff; c.min_side = self.min_side; c.max_side = self.max_side
        c.dynamic_rt = int(self.dynamic_rt)
        c.unsplit = int(self.unsplit)
        return c


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_H = ctypes.c_void_p

# int (*)(void* ctx, int level, int kind): the exchange hook of a partitioned hierarchy
_HOOK = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int)
# exchange kinds (MLSWE_XCHG_*)
XCHG_FULL, XCHG_HALO, XCHG_LAST, XCHG_AVERAGED = 0, 1, 2, 3

# name -> argtypes (restype is mlswe_status unless stated)
_SIGS = {
    "mlswe_create_hierarchy": [ctypes.POINTER(_Config), ctypes.c_int, ctypes.POINTER(_Domain),
                               ctypes.POINTER(_Allocator), ctypes.c_void_p, ctypes.POINTER(_H)],
    "mlswe_destroy": [_H],
    "mlswe_level_shape": [_H, ctypes.c_int, ctypes.c_int, _ip, _ip],
    "mlswe_set_bathymetry": [_H, ctypes.c_int, _dp],
    "mlswe_get_bathymetry": [_H, ctypes.c_int, ctypes.c_int, _dp],
    "mlswe_set_state": [_H, ctypes.c_int, ctypes.c_int, _dp],
    "mlswe_set_state_async": [_H, ctypes.c_int, ctypes.c_int, _dp],
    "mlswe_get_rows_device": [_H, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p],
    "mlswe_set_rows_device": [_H, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p],
    "mlswe_read_gauges_async": [_H, ctypes.c_int, ctypes.c_int, _dp, _dp],
    "mlswe_synchronize": [_H],
    "mlswe_get_state": [_H, ctypes.c_int, ctypes.c_int, _dp],
    "mlswe_set_patches": [_H, ctypes.c_int, ctypes.c_int, ctypes.c_int, _i32p],
    "mlswe_get_patches": [_H, ctypes.c_int, ctypes.c_int, _ip, _i32p],
    "mlswe_set_dt": [_H, ctypes.c_int, _dp],
    "mlswe_step_level": [_H, ctypes.c_int, _dp, _dp],
    "mlswe_fill_ghosts": [_H, ctypes.c_int, ctypes.c_double],
    "mlswe_interp_fine": [_H, ctypes.c_int, ctypes.c_int],
    "mlswe_average_coarse": [_H, ctypes.c_int, ctypes.c_int],
    "mlswe_get_flags": [_H, ctypes.c_int, ctypes.c_int, _u8p],
    "mlswe_regrid": [_H, ctypes.c_int],
    "mlswe_advance": [_H, ctypes.c_int],
    "mlswe_get_time": [_H, _dp, _dp],
    "mlswe_read_gauges": [_H, ctypes.c_int, ctypes.c_int, _dp, _dp],
    "mlswe_set_tiles": [_H, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int],
    "mlswe_set_execution": [_H, ctypes.c_int, ctypes.c_int],
    "mlswe_adjoint_setup": [_H, ctypes.c_int, ctypes.c_int, ctypes.c_int, _i32p, _dp],
    "mlswe_adjoint_keep_edge_data": [_H, ctypes.c_int],
    "mlswe_hyperbolicity_losses": [_H, ctypes.POINTER(ctypes.c_longlong), ctypes.c_int],
    "mlswe_get_clock": [_H, _dp, ctypes.c_int],
    "mlswe_get_stats": [_H, ctypes.c_void_p],
    "mlswe_set_clock": [_H, _dp, ctypes.c_int],
    "mlswe_fixed_set_controls": [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double],
    "mlswe_fixed_forward": [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, _dp],
    "mlswe_fixed_forward_state": [_H, _dp],
    "mlswe_fixed_backward": [_H, ctypes.c_void_p, ctypes.c_void_p],
    "mlswe_fixed_backward_state": [_H, ctypes.c_void_p, ctypes.c_void_p],
    "mlswe_autotune": [_H, ctypes.c_int, ctypes.c_int, _ip],
    "mlswe_set_partition": [_H, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p],
    "mlswe_partition_owners": [_H, ctypes.c_int, ctypes.c_int, _ip],
    "mlswe_partition_sizes": [_H, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong)],
    "mlswe_partition_pack": [_H, ctypes.c_int, ctypes.c_int, ctypes.c_void_p],
    "mlswe_partition_unpack": [_H, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p],
    "mlswe_wave_speed_slots": [_H, ctypes.POINTER(ctypes.c_void_p), _ip],
    "mlswe_timing": [_H, ctypes.c_int, ctypes.c_int, _dp, ctypes.POINTER(ctypes.c_longlong),
                     ctypes.POINTER(ctypes.c_longlong)],
}

KERNEL_CLASSES = ["sweep_x", "sweep_y", "ghost_fill", "interp_fine", "average", "flags", "reflux", "other",
                  "adjoint", "update"]


def build(force: bool = False) -> str:
    """Compile the CUDA library for sm_103a (in tree)."""
    return _build_mod.build(force=force)


def lib():
    """Load the CUDA library; raises if it is missing (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise MLSWEError(9, f"CUDA library not built: {LIB_PATH} (run paper_1803_01450_gb300.build())")
    L = ctypes.CDLL(LIB_PATH)
    for name, args in _SIGS.items():
        fn = getattr(L, name, None)
        if fn is None:
            continue
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.mlswe_last_error.argtypes = [_H]
    L.mlswe_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def exported_symbols() -> list:
    L = lib()
    return [n for n in list(_SIGS) + ["mlswe_last_error"] if hasattr(L, n)]


def _d(a: np.ndarray):
    return a.ctypes.data_as(_dp)


class _Stats(ctypes.Structure):
    _fields_ = [("coarse_steps", ctypes.c_longlong), ("regrids", ctypes.c_longlong),
                ("level_steps", ctypes.c_longlong * 4), ("cell_updates", ctypes.c_longlong * 4),
                ("patches", ctypes.c_int * 4), ("cfl_exceeded", ctypes.c_longlong), ("last_cfl", ctypes.c_double)]


def _python_allocator(alloc, free):
    """Allocator callback from two Python callables: alloc(nbytes) -> device pointer (int;
    0 or None on failure) and free(pointer)."""

    def _alloc(nbytes, stream, ctx):
        try:
            return alloc(int(nbytes)) or None
        except Exception:
            return None

    def _free(ptr, stream, ctx):
        free(ptr)

    return _Allocator(_ALLOC_FN(_alloc), _FREE_FN(_free), None)


def _torch_allocator():
    import torch

    dev = torch.cuda.current_device()

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream or 0)
        except Exception:
            return None

    def _free(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    a = _Allocator(_ALLOC_FN(_alloc), _FREE_FN(_free), None)
    return a


class Hierarchy:
    """A set of ensemble members, each a hierarchy of refinement levels (C ABI handle)."""

    def __init__(self, cfg: Config, domains: Sequence[tuple], stream: Optional[int] = None,
                 use_torch_allocator: bool = True, allocator=None):
        """allocator: optional (alloc, free) pair of callables (alloc(nbytes) -> device pointer
        or 0, free(pointer)) used instead of torch's caching allocator."""
        self.cfg = cfg
        self.L = lib()
        self._pending = []  # host arrays of asynchronous copies, kept alive until synchronize()
        doms = (_Domain * len(domains))()
        for k, d in enumerate(domains):
            x0, y0, x1, y1, nx0, ny0 = d
            doms[k] = _Domain(x0, y0, x1, y1, nx0, ny0)
        self._c_cfg = cfg.to_c()
        self._alloc = None
        alloc_ptr = None
        if allocator is not None:
            self._alloc = _python_allocator(*allocator)
            alloc_ptr = ctypes.byref(self._alloc)
        elif use_torch_allocator:
            import torch
            if not torch.cuda.is_available():
                raise MLSWEError(9, "no CUDA device")
            self._alloc = _torch_allocator()
            alloc_ptr = ctypes.byref(self._alloc)
            if stream is None:
                stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        h = _H()
        st = self.L.mlswe_create_hierarchy(ctypes.byref(self._c_cfg), len(domains), doms, alloc_ptr,
                                           ctypes.c_void_p(stream or 0), ctypes.byref(h))
        if st != MLSWE_OK:
            raise MLSWEError(st, "mlswe_create_hierarchy failed")
        self.h = h
        self.n_members = len(domains)
        self.M = cfg.M

    def _check(self, st: int, what: str, ok=(MLSWE_OK,)):
        if st not in ok:
            raise MLSWEError(st, f"{what}: {self.L.mlswe_last_error(self.h).decode()}")
        return st

    def close(self):
        if getattr(self, "h", None):
            self.L.mlswe_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def shape(self, member: int, level: int):
        nx, ny = ctypes.c_int(), ctypes.c_int()
        self._check(self.L.mlswe_level_shape(self.h, member, level, ctypes.byref(nx), ctypes.byref(ny)), "level_shape")
        return ny.value, nx.value

    def set_bathymetry(self, member: int, B_finest: np.ndarray):
        B = np.ascontiguousarray(B_finest, dtype=np.float64)
        self._check(self.L.mlswe_set_bathymetry(self.h, member, _d(B)), "set_bathymetry")

    def get_bathymetry(self, member: int, level: int) -> np.ndarray:
        ny, nx = self.shape(member, level)
        out = np.zeros((ny, nx))
        self._check(self.L.mlswe_get_bathymetry(self.h, member, level, _d(out)), "get_bathymetry")
        return out

    def set_state(self, member: int, level: int, q: np.ndarray):
        q = np.ascontiguousarray(q, dtype=np.float64)
        ny, nx = self.shape(member, level)
        assert q.shape == (3 * self.M, ny, nx), q.shape
        self._check(self.L.mlswe_set_state(self.h, member, level, _d(q)), "set_state")

    def set_state_async(self, member: int, level: int, q: np.ndarray):
        """Enqueues q (page-locked for the copy to overlap running work) as the state of
        (member, level) after the work already enqueued; q is kept alive and must stay
        unchanged until synchronize()."""
        ny, nx = self.shape(member, level)
        if not (q.dtype == np.float64 and q.flags.c_contiguous and q.shape == (3 * self.M, ny, nx)):
            raise MLSWEError(1, "set_state_async: q must be a C-contiguous float64 [3M][ny][nx] array")
        self._pending.append(q)
        self._check(self.L.mlswe_set_state_async(self.h, member, level, _d(q)), "set_state_async")

    def read_gauges_async(self, member: int, xy: np.ndarray, out: np.ndarray):
        """Enqueues the gauge read into out ([n][M] float64, page-locked for an asynchronous
        copy); the values are there after synchronize()."""
        xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
        if not (out.dtype == np.float64 and out.flags.c_contiguous and out.shape == (len(xy), self.M)):
            raise MLSWEError(1, "read_gauges_async: out must be a C-contiguous float64 [n][M] array")
        self._pending.append(out)
        self._check(self.L.mlswe_read_gauges_async(self.h, member, len(xy), _d(xy), _d(out)), "read_gauges_async")

    def synchronize(self):
        self._check(self.L.mlswe_synchronize(self.h), "synchronize")
        self._pending.clear()

    def get_state(self, member: int, level: int) -> np.ndarray:
        ny, nx = self.shape(member, level)
        out = np.zeros((3 * self.M, ny, nx))
        self._check(self.L.mlswe_get_state(self.h, member, level, _d(out)), "get_state")
        return out

    def set_patches(self, member: int, level: int, boxes):
        b = np.ascontiguousarray(np.asarray(boxes, dtype=np.int32).reshape(-1, 4))
        return self._check(self.L.mlswe_set_patches(self.h, member, level, len(b), b.ctypes.data_as(_i32p)),
                           "set_patches")

    def get_patches(self, member: int, level: int) -> np.ndarray:
        n = ctypes.c_int(0)
        self._check(self.L.mlswe_get_patches(self.h, member, level, ctypes.byref(n), None), "get_patches")
        out = np.zeros((max(n.value, 1), 4), dtype=np.int32)
        cap = ctypes.c_int(n.value)
        self._check(self.L.mlswe_get_patches(self.h, member, level, ctypes.byref(cap), out.ctypes.data_as(_i32p)),
                    "get_patches")
        return out[: n.value]

    def set_dt(self, level: int, dt):
        dt = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, float), (self.n_members,)))
        self._check(self.L.mlswe_set_dt(self.h, level, _d(dt)), "set_dt")

    def step_level(self, level: int, dt=None, want_cfl: bool = False, allow=(MLSWE_OK,)):
        dtp = None
        if dt is not None:
            dta = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, float), (self.n_members,)))
            dtp = _d(dta)
        cfl = np.zeros(self.n_members) if want_cfl else None
        self._check(self.L.mlswe_step_level(self.h, level, dtp, _d(cfl) if want_cfl else None), "step_level", allow)
        return cfl

    def fill_ghosts(self, level: int, alpha: float):
        self._check(self.L.mlswe_fill_ghosts(self.h, level, float(alpha)), "fill_ghosts")

    def interp_fine(self, coarse_level: int, member: int):
        self._check(self.L.mlswe_interp_fine(self.h, coarse_level, member), "interp_fine")

    def average_coarse(self, fine_level: int, member: int):
        self._check(self.L.mlswe_average_coarse(self.h, fine_level, member), "average_coarse")

    def get_flags(self, member: int, level: int) -> np.ndarray:
        ny, nx = self.shape(member, level)
        out = np.zeros((ny, nx), dtype=np.uint8)
        self._check(self.L.mlswe_get_flags(self.h, member, level, out.ctypes.data_as(_u8p)), "get_flags")
        return out

    def regrid(self, base_level: int = 0):
        self._check(self.L.mlswe_regrid(self.h, base_level), "regrid")

    def advance(self, n_coarse_steps: int, allow=(MLSWE_OK,)):
        st = self.L.mlswe_advance(self.h, n_coarse_steps)
        err = getattr(self, "_hook_error", None)
        if err is not None:
            self._hook_error = None
            raise MLSWEError(st, f"advance: the exchange hook raised {err!r}") from err
        return self._check(st, "advance", allow)

    # ---- patch partition across ranks (mlswe_set_partition and the exchange calls) ----
    def set_partition(self, rank: int, world_size: int, hook=None):
        """Sweep only this rank's patches of the refined levels; hook(level, kind), if given,
        is called by advance at the exchange points (kind: XCHG_FULL, XCHG_HALO, XCHG_LAST,
        XCHG_AVERAGED) and must exchange (see sharding)."""
        cb = None
        if hook is not None:
            def _cb(ctx, level, kind):
                try:
                    hook(level, kind)
                    return 0
                except BaseException as e:  # reported by advance
                    self._hook_error = e
                    return 1
            cb = _HOOK(_cb)
        self._hook_ref = cb  # the C side keeps only the function pointer
        self._hook_error = None
        fp = ctypes.cast(cb, ctypes.c_void_p) if cb is not None else None
        self._check(self.L.mlswe_set_partition(self.h, rank, world_size, fp, None), "set_partition")
        self.part_rank, self.part_size = rank, world_size

    def partition_owners(self, member: int, level: int) -> np.ndarray:
        out = np.zeros(len(self.get_patches(member, level)), dtype=np.int32)
        self._check(self.L.mlswe_partition_owners(self.h, member, level,
                                                  out.ctypes.data_as(ctypes.POINTER(ctypes.c_int))),
                    "partition_owners")
        return out

    def partition_sizes(self, level: int, kind: int = 0):
        """Doubles in every rank's packed buffer of `level` and exchange `kind`."""
        n = getattr(self, "part_size", 1)
        out = (ctypes.c_longlong * n)()
        self._check(self.L.mlswe_partition_sizes(self.h, level, int(kind), out), "partition_sizes")
        return [int(v) for v in out]

    def partition_pack(self, level: int, dst_ptr: int, kind: int = 0):
        self._check(self.L.mlswe_partition_pack(self.h, level, int(kind), ctypes.c_void_p(dst_ptr)),
                    "partition_pack")

    def partition_unpack(self, level: int, rank: int, src_ptr: int, kind: int = 0):
        self._check(self.L.mlswe_partition_unpack(self.h, level, int(kind), rank, ctypes.c_void_p(src_ptr)),
                    "partition_unpack")

    def wave_speed_slots(self):
        """(device address, count) of the wave-speed slots (float64, non-negative)."""
        p, n = ctypes.c_void_p(), ctypes.c_int()
        self._check(self.L.mlswe_wave_speed_slots(self.h, ctypes.byref(p), ctypes.byref(n)), "wave_speed_slots")
        return int(p.value), int(n.value)

    def get_time(self):
        """(simulated time per member, next level-0 time step per member)."""
        t = np.zeros(self.n_members)
        dt = np.zeros(self.n_members)
        self._check(self.L.mlswe_get_time(self.h, _d(t), _d(dt)), "get_time")
        return t, dt

    def set_execution(self, use_graphs: bool = True, per_patch_launches: bool = False):
        self._check(self.L.mlswe_set_execution(self.h, int(use_graphs), int(per_patch_launches)), "set_execution")

    def autotune(self, level: int, iters: int = 5):
        out = (ctypes.c_int * 6)()
        self._check(self.L.mlswe_autotune(self.h, level, iters, out), "autotune")
        return tuple(out)

    def set_tiles(self, dir: int, length: int, lines: int, ctas_per_sm: int = 1):
        self._check(self.L.mlswe_set_tiles(self.h, dir, length, lines, ctas_per_sm), "set_tiles")

    def adjoint_setup(self, n_steps: int, ckpt_every: int, gauge_ij: np.ndarray, obs: np.ndarray):
        g = np.ascontiguousarray(np.asarray(gauge_ij, dtype=np.int32).reshape(-1, 2))
        o = np.ascontiguousarray(np.asarray(obs, dtype=np.float64).reshape(n_steps, len(g)))
        self._check(self.L.mlswe_adjoint_setup(self.h, n_steps, ckpt_every, len(g), g.ctypes.data_as(_i32p), _d(o)),
                    "adjoint_setup")

    def get_stats(self) -> dict:
        """Run counters: coarse steps, regrids, per-level steps, cell updates and patch counts,
        member coarse steps above cfl_max, the last Courant number."""
        st = _Stats()
        self._check(self.L.mlswe_get_stats(self.h, ctypes.cast(ctypes.byref(st), ctypes.c_void_p)), "get_stats")
        L = self.cfg.max_levels
        return {"coarse_steps": st.coarse_steps, "regrids": st.regrids,
                "level_steps": list(st.level_steps)[:L], "cell_updates": list(st.cell_updates)[:L],
                "patches": list(st.patches)[:L], "cfl_exceeded": st.cfl_exceeded, "last_cfl": st.last_cfl}

    def clock_size(self) -> int:
        return self.n_members * (1 + 3 * self.cfg.max_levels) + 3

    def get_clock(self) -> np.ndarray:
        """Time-stepping state (member times, next-step wave speeds, step counter) for resume."""
        buf = np.zeros(self.clock_size())
        self._check(self.L.mlswe_get_clock(self.h, _d(buf), len(buf)), "get_clock")
        return buf

    def set_clock(self, buf: np.ndarray):
        """Restores get_clock()'s record; call it after the last set_state."""
        b = np.ascontiguousarray(buf, dtype=np.float64)
        self._check(self.L.mlswe_set_clock(self.h, _d(b), len(b)), "set_clock")

    def hyperbolicity_losses(self, reset: bool = True) -> int:
        """Edges that used the eigenvalue guesses (loss of hyperbolicity) since the last reset."""
        c = ctypes.c_longlong(0)
        self._check(self.L.mlswe_hyperbolicity_losses(self.h, ctypes.byref(c), 1 if reset else 0),
                    "hyperbolicity_losses")
        return c.value

    def adjoint_keep_edge_data(self, enable: bool = True):
        """Keep per-edge forward records of the recomputed steps (default) or rebuild them in
        the transposed sweeps; takes effect at the next adjoint_setup."""
        self._check(self.L.mlswe_adjoint_keep_edge_data(self.h, 1 if enable else 0), "adjoint_keep_edge_data")

    def get_rows_device(self, member: int, level: int, j0: int, n: int, dst_ptr: int):
        """Rows [j0, j0 + n) of the level's state into a device buffer [3M][n][nx] (stream-ordered)."""
        self._check(self.L.mlswe_get_rows_device(self.h, member, level, j0, n, ctypes.c_void_p(dst_ptr)),
                    "get_rows_device")

    def set_rows_device(self, member: int, level: int, j0: int, n: int, src_ptr: int):
        """A device buffer [3M][n][nx] into rows [j0, j0 + n) of the level's state (stream-ordered)."""
        self._check(self.L.mlswe_set_rows_device(self.h, member, level, j0, n, ctypes.c_void_p(src_ptr)),
                    "set_rows_device")

    def fixed_set_controls(self, eta1_ptr: int, B_ptr: int, eta2: float):
        """Initial state of the gauge-misfit problem from the device controls eta_1(0), B."""
        self._check(self.L.mlswe_fixed_set_controls(self.h, ctypes.c_void_p(eta1_ptr), ctypes.c_void_p(B_ptr),
                                                    float(eta2)), "fixed_set_controls")

    def fixed_forward(self, eta1_ptr: int, B_ptr: int, eta2: float) -> float:
        """Loss of the forward pass from the device controls eta_1(0), B ([ny][nx] each)."""
        loss = ctypes.c_double(0.0)
        self._check(self.L.mlswe_fixed_forward(self.h, ctypes.c_void_p(eta1_ptr), ctypes.c_void_p(B_ptr),
                                               float(eta2), ctypes.byref(loss)), "fixed_forward")
        return loss.value

    def fixed_forward_state(self) -> float:
        """Loss of the forward pass from the current state."""
        loss = ctypes.c_double(0.0)
        self._check(self.L.mlswe_fixed_forward_state(self.h, ctypes.byref(loss)), "fixed_forward_state")
        return loss.value

    def fixed_backward(self, d_eta1_ptr: int, dB_ptr: int):
        """Writes dJ/d eta_1(0) and dJ/dB ([ny][nx] each) into caller-owned device buffers."""
        self._check(self.L.mlswe_fixed_backward(self.h, ctypes.c_void_p(d_eta1_ptr), ctypes.c_void_p(dB_ptr)),
                    "fixed_backward")

    def fixed_backward_state(self, dq0_ptr: int, dB_ptr: int):
        """Writes dJ/dQ^0 ([3M][ny][nx]) and dJ/dB at fixed Q^0 ([ny][nx]) into caller-owned
        device buffers."""
        self._check(self.L.mlswe_fixed_backward_state(self.h, ctypes.c_void_p(dq0_ptr), ctypes.c_void_p(dB_ptr)),
                    "fixed_backward_state")

    def timing(self, enable: bool = True):
        """Per-kernel-class device time (ms) and launches since the last call; resets them."""
        n = len(KERNEL_CLASSES)
        ms = np.zeros(n)
        cnt = (ctypes.c_longlong * n)()
        tot = ctypes.c_longlong(0)
        self._check(self.L.mlswe_timing(self.h, int(enable), n, _d(ms), cnt, ctypes.byref(tot)), "timing")
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KERNEL_CLASSES)}, int(tot.value)

    def read_gauges(self, member: int, xy: np.ndarray) -> np.ndarray:
        xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
        out = np.zeros((len(xy), self.M))
        self._check(self.L.mlswe_read_gauges(self.h, member, len(xy), _d(xy), _d(out)), "read_gauges")
        return out
