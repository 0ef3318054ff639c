"""Work split across GPUs (one process per GPU, torch.distributed): host-side bookkeeping only.

Two splits of the method's work, both without changing a single arithmetic operation of a
member's step:

* Ensemble members are independent problems. partition_members assigns whole members to
  ranks, largest first to the least-loaded rank (by cells per coarse step); a rank builds one
  hierarchy over its members and advances them in its own batched launches. Only scalars
  cross ranks (cell updates, times), through all-reduces.
* One grid split into slabs of rows. A rank holds its rows plus two halo rows on each side
  that faces another slab (at the domain's own walls the slab keeps the wall). Before every
  step the ranks swap the two rows next to each shared slab edge; the x sweep then runs over
  every local row (halo rows included: their rows are complete in x) and the y sweep updates
  the owned rows from cells at most two rows away, all of them local and current. The rows a
  rank owns therefore come out exactly as in the undivided grid. The rows beyond a halo (the
  local array's end, which the solver treats as a wall) only ever feed the halo rows, which
  the next swap overwrites. A time step common to all slabs is the minimum over the ranks
  (min_all).

* The patches of an AMR hierarchy's refined levels split over the ranks. Every rank holds
  the whole hierarchy; the library sweeps only the rank's own patches of the levels >= 1
  (owners by a space-filling curve, partition_patches restates the rule) and calls a hook
  after every refined level step, in which the ranks all-gather their packed patch values
  and take the maximum of the wave-speed slots (exchange_level; PatchPartition wires it to
  a Hierarchy). Level 0, ghost fill, coarsening, reflux, time steps and regrids run on
  every rank, so every rank's hierarchy equals the undivided one. The finest level moves
  less: between its substeps only the halo cells (the cells of a rank's patches within two
  cells of another rank's patch), after the last one the halo cells and the reflux
  accumulators; each rank coarsens its own finest patches and sends the parent cells under
  them; the whole finest level moves only before a regrid and at the end of an advance.

Data moves only by point-to-point sends or all-gathers into local buffers and by
all-reduces (NCCL on GPUs, gloo on CPUs); the stepping itself is a callable the caller
supplies (the CUDA library's level step) or the library's own driver.
"""
from __future__ import annotations

from dataclasses import dataclass

HALO = 2  # rows each side of a shared slab edge: the second-order stencil reaches two cells


def partition_members(costs, world_size):
    """Member indices per rank: members in decreasing cost (ties: lower index first), each to
    the rank with the least cost so far (ties: lower rank); each rank's list in index order."""
    order = sorted(range(len(costs)), key=lambda k: (-costs[k], k))
    load = [0] * world_size
    out = [[] for _ in range(world_size)]
    for k in order:
        r = min(range(world_size), key=lambda j: (load[j], j))
        out[r].append(k)
        load[r] += costs[k]
    return [sorted(v) for v in out]


@dataclass(frozen=True)
class Slab:
    """Rows [j0, j1) of an ny-row grid owned by a rank; local rows [lo, hi) held (halos)."""
    j0: int
    j1: int
    lo: int
    hi: int

    @property
    def rows(self) -> int:
        return self.hi - self.lo

    @property
    def own(self) -> slice:
        """The owned rows as a slice of the local array."""
        return slice(self.j0 - self.lo, self.j1 - self.lo)


def slab_of(ny, world_size, rank):
    """Even split of ny rows (the first ny % world_size ranks take one more); each slab must
    own at least HALO rows so that its neighbour's halo lies in it."""
    base, extra = divmod(ny, world_size)
    if base < HALO:
        raise ValueError(f"{ny} rows cannot be split into {world_size} slabs of at least {HALO} rows")
    j0 = rank * base + min(rank, extra)
    j1 = j0 + base + (1 if rank < extra else 0)
    lo = j0 - HALO if rank > 0 else 0
    hi = j1 + HALO if rank < world_size - 1 else ny
    return Slab(j0, j1, lo, hi)


def halo_exchange(slab: Slab, rank, world_size, get_rows, set_rows, dist, group=None):
    """Swaps the HALO rows next to every shared slab edge with the neighbouring ranks.

    get_rows(r0, n) returns the local rows [r0, r0 + n) as a contiguous tensor (every field);
    set_rows(r0, n, t) writes such a tensor back. Sends go out and receives come in as one
    batch of point-to-point operations, so neither neighbour waits for the other to finish."""
    ops, recv = [], []
    if rank > 0:
        send_lo = get_rows(slab.j0 - slab.lo, HALO)
        buf_lo = send_lo.new_empty(send_lo.shape)
        ops += [dist.P2POp(dist.isend, send_lo, rank - 1, group), dist.P2POp(dist.irecv, buf_lo, rank - 1, group)]
        recv.append((0, buf_lo))
    if rank < world_size - 1:
        send_hi = get_rows(slab.j1 - slab.lo - HALO, HALO)
        buf_hi = send_hi.new_empty(send_hi.shape)
        ops += [dist.P2POp(dist.isend, send_hi, rank + 1, group), dist.P2POp(dist.irecv, buf_hi, rank + 1, group)]
        recv.append((slab.j1 - slab.lo, buf_hi))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    for r0, buf in recv:
        set_rows(r0, HALO, buf)


def _reduce(value, op, dist, device):
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t.item())


def sum_all(value, dist, device=None):
    return _reduce(value, dist.ReduceOp.SUM, dist, device)


def max_all(value, dist, device=None):
    return _reduce(value, dist.ReduceOp.MAX, dist, device)


def min_all(value, dist, device=None):
    return _reduce(value, dist.ReduceOp.MIN, dist, device)


# ---------------------------------------------------------------------- patch partition
def morton(i: int, j: int) -> int:
    """Z-order key of a cell index pair: the low 21 bits of i in the even bits, of j in the
    odd bits."""
    key = 0
    for b in range(21):
        key |= ((i >> b) & 1) << (2 * b)
        key |= ((j >> b) & 1) << (2 * b + 1)
    return key


def partition_patches(layouts, world_size):
    """Owner rank of every patch of one refined level over all members (layouts: per member an
    (n, 4) array of boxes i0, j0, i1, j1). Patches in order of member, then Morton key of the
    integer centre ((i0 + i1) // 2, (j0 + j1) // 2), then index; with T the cells of all of
    them and c the cells before a patch, the patch goes to min(n - 1, (2 c + cells) n // (2 T)):
    the rank whose share of the cells holds the patch's middle cell."""
    entries = []
    for m, boxes in enumerate(layouts):
        for p, (i0, j0, i1, j1) in enumerate(boxes):
            entries.append((m, morton((i0 + i1) // 2, (j0 + j1) // 2), p, (i1 - i0) * (j1 - j0)))
    entries.sort()
    total = sum(e[3] for e in entries)
    owners = [[0] * len(b) for b in layouts]
    before = 0
    for m, _, p, cells in entries:
        r = min(world_size - 1, (2 * before + cells) * world_size // (2 * total)) if total > 0 else 0
        owners[m][p] = r
        before += cells
    return owners


def exchange_level(rank, world_size, sizes, pack, unpack, speeds, dist, new_buffer):
    """The exchange after a refined level step: every rank packs its patches into a buffer of
    max(sizes) values (pack(buf)), the buffers are all-gathered, each rank writes the other
    ranks' patches (unpack(q, buf_q) for q != rank with sizes[q] > 0), and the wave-speed
    slots become their maximum over the ranks (speeds: a float64 tensor, or None)."""
    n = max(sizes) if sizes else 0
    if n > 0:
        send = new_buffer(n)
        pack(send)
        recv = [new_buffer(n) for _ in range(world_size)]
        dist.all_gather(recv, send)
        for q in range(world_size):
            if q != rank and sizes[q] > 0:
                unpack(q, recv[q])
    if speeds is not None:
        dist.all_reduce(speeds, op=dist.ReduceOp.MAX)


class _DeviceArray:
    """A float64 device array the library owns, seen by torch without a copy."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f8", "data": (ptr, False), "version": 2}


class PatchPartition:
    """Partition of a Hierarchy's refined-level patches over the ranks of a process group
    (NCCL): sets the hierarchy's partition and the exchange hook that mlswe_advance calls.
    The collectives run on the hierarchy's stream, ordered with its kernels."""

    def __init__(self, H, rank, world_size, dist, device):
        self.H, self.rank, self.ws, self.dist, self.device = H, rank, world_size, dist, device
        H.set_partition(rank, world_size, self._exchange)

    def _exchange(self, level, kind):
        import torch
        H = self.H
        stream = torch.cuda.ExternalStream(H.stream, device=self.device)
        with torch.cuda.stream(stream):
            ptr, n = H.wave_speed_slots()
            # the speeds' maximum is idempotent: taken at every kind of exchange
            speeds = torch.as_tensor(_DeviceArray(ptr, n), device=self.device)
            exchange_level(self.rank, self.ws, H.partition_sizes(level, kind),
                           lambda buf: H.partition_pack(level, buf.data_ptr(), kind),
                           lambda q, buf: H.partition_unpack(level, q, buf.data_ptr(), kind),
                           speeds, self.dist,
                           lambda k: torch.empty(k, dtype=torch.float64, device=self.device))
