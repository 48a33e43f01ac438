"""z-slab decomposition of the PPML step over ranks (one GPU per rank).

The grid's z planes are split into contiguous slabs, one per rank.  A slab's state lives in
arrays padded by PPML_HALO_PLANES planes behind every z face it shares with another slab
(both faces of every slab on a periodic z axis); the kernels read those planes like interior
cells (boundary type PPML_BC_HALO), and the whole grid's own z boundaries stay on the outer
slabs.  One step (the order of the paper's scheme, Sec. 1, with the two exchanges its
stencils need):

  1. the halo planes of U^n from the neighbours;
  2. the Eulerian stage of the slab (S1-S3) into the slab's U*;
  3. the halo planes of U* from the neighbours;
  4. the Lagrangian stage, energy correction and the slab's CFL maxima and FP64 sums;
  5. an all-reduce of those (max of the two maxima, sum of the sums and counts);
  6. the time, the next CFL step (Sec. 1.1) and the diagnostics from the reduced values.

The stages and the reduced scalars run in libppml's kernels (a ``Stages`` object: the
library's slab calls); this module only moves planes and reduces ten numbers.  The
exchange and the all-reduce use ``torch.distributed`` (NCCL between GPUs, gloo between
CPU processes), or, for several slabs driven by one process on one device, direct copies
(``LocalComm``).  Every cell takes the same operations on the same values as on one grid,
so the decomposed state equals the single grid's bit for bit.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

HALO_PLANES = 3
REDUCE_LEN = 10
TILE = 16  # z planes of a stage kernel's tile
OUTFLOW, PERIODIC, REFLECT, HALO = 0, 1, 2, 3


def slab_bounds(nz, world):
    """First plane of every slab and nz: boundaries on tile boundaries (multiples of TILE)
    nearest to an even split, so that every cell sits at the same place in its tile as on
    one grid and FP32 results agree bit for bit too; an even split of the planes where that
    leaves a slab with fewer than HALO_PLANES planes (FP64 still agrees bit for bit, FP32 to
    rounding: the kernels' FMA contraction may differ between places in a tile)."""
    aligned = [TILE * round(r * nz / (TILE * world)) for r in range(world)] + [nz]
    if all(b - a >= HALO_PLANES for a, b in zip(aligned, aligned[1:])):
        return aligned
    base, extra = divmod(nz, world)
    return [r * base + min(r, extra) for r in range(world)] + [nz]


@dataclass
class SlabLayout:
    """Rank `rank` of `world`'s share of a grid of n = (nx, ny, nz) cells with boundaries
    bc (-x, +x, -y, +y, -z, +z): planes [z0, z0 + nz) of the whole grid."""
    n: tuple
    bc: tuple
    world: int
    rank: int

    def __post_init__(self):
        nx, ny, nz = (int(v) for v in self.n)
        if not 0 <= self.rank < self.world:
            raise ValueError("rank out of range")
        bounds = slab_bounds(nz, self.world)
        self.z0 = bounds[self.rank]
        self.nz = bounds[self.rank + 1] - bounds[self.rank]
        self.tile_aligned = all(b % TILE == 0 for b in bounds[:-1])
        if self.world > 1 and self.nz < HALO_PLANES:
            raise ValueError(f"slab of {self.nz} planes: each needs at least {HALO_PLANES}")
        periodic = self.bc[4] == PERIODIC
        self.lo_halo = self.world > 1 and (self.rank > 0 or periodic)
        self.hi_halo = self.world > 1 and (self.rank < self.world - 1 or periodic)
        self.slab_bc = tuple(self.bc[:4]) + (HALO if self.lo_halo else self.bc[4],
                                             HALO if self.hi_halo else self.bc[5])
        self.lo_nb = (self.rank - 1) % self.world
        self.hi_nb = (self.rank + 1) % self.world
        self.plane = nx * ny
        self.pad_lo = HALO_PLANES if self.lo_halo else 0
        self.pad_hi = HALO_PLANES if self.hi_halo else 0
        self.planes = self.pad_lo + self.nz + self.pad_hi
        self.slab_n = (nx, ny, self.nz)

    @property
    def cells(self) -> int:
        return self.plane * self.nz

    def interior(self, t):
        """The slab's own planes of a padded field (a view)."""
        return t[self.pad_lo * self.plane:(self.pad_lo + self.nz) * self.plane]

    # contiguous plane blocks of a padded field
    def send_down(self, t):  # the slab's first planes, to the neighbour below
        return t[self.pad_lo * self.plane:(self.pad_lo + HALO_PLANES) * self.plane]

    def send_up(self, t):  # the slab's last planes, to the neighbour above
        e = (self.pad_lo + self.nz) * self.plane
        return t[e - HALO_PLANES * self.plane:e]

    def halo_lo(self, t):
        return t[:self.pad_lo * self.plane]

    def halo_hi(self, t):
        e = (self.pad_lo + self.nz) * self.plane
        return t[e:e + self.pad_hi * self.plane]


class DistComm:
    """Halo exchange and all-reduce between ranks through torch.distributed."""

    def __init__(self, dist, layout: SlabLayout):
        self.dist = dist
        self.L = layout

    def exchange(self, fields):
        """Every slab's first planes go down (into the upper halo of the slab below), then
        its last planes go up.  Per pair of ranks the sends and receives come in the same
        order (all downward transfers first), as NCCL, which ignores tags, needs when one
        neighbour is both below and above (two slabs on a periodic axis)."""
        L, d = self.L, self.dist
        if L.world == 1:
            return
        ops = []
        for f, t in enumerate(fields):  # downward: tag 2f
            if L.lo_halo:
                ops.append(d.P2POp(d.isend, L.send_down(t), L.lo_nb, tag=2 * f))
        for f, t in enumerate(fields):
            if L.hi_halo:
                ops.append(d.P2POp(d.irecv, L.halo_hi(t), L.hi_nb, tag=2 * f))
        for f, t in enumerate(fields):  # upward: tag 2f + 1
            if L.hi_halo:
                ops.append(d.P2POp(d.isend, L.send_up(t), L.hi_nb, tag=2 * f + 1))
        for f, t in enumerate(fields):
            if L.lo_halo:
                ops.append(d.P2POp(d.irecv, L.halo_lo(t), L.lo_nb, tag=2 * f + 1))
        if ops:
            for r in d.batch_isend_irecv(ops):
                r.wait()

    def allreduce(self, red):
        if self.L.world == 1:
            return
        self.dist.all_reduce(red[:2], op=self.dist.ReduceOp.MAX)
        self.dist.all_reduce(red[2:], op=self.dist.ReduceOp.SUM)


class LocalComm:
    """The same exchange and all-reduce for all slabs of a grid driven by one process
    (one device): plane copies between the slabs' arrays; the maxima and sums over the
    slabs' reduce buffers in rank order."""

    def __init__(self, layouts):
        self.layouts = layouts

    def exchange(self, fields_by_rank):
        Ls = self.layouts
        for r, L in enumerate(Ls):
            for f, t in enumerate(fields_by_rank[r]):
                if L.lo_halo:
                    L.halo_lo(t).copy_(Ls[L.lo_nb].send_up(fields_by_rank[L.lo_nb][f]))
                if L.hi_halo:
                    L.halo_hi(t).copy_(Ls[L.hi_nb].send_down(fields_by_rank[L.hi_nb][f]))

    def allreduce(self, reds):
        tot = reds[0].clone()
        for r in reds[1:]:
            tot[:2] = torch.maximum(tot[:2], r[:2])
            tot[2:] += r[2:]
        for r in reds:
            r.copy_(tot)


class Stages:
    """libppml's slab calls for one slab: a grid handle over the slab's interior planes with
    halo faces, and the padded state, U* and output arrays."""

    def __init__(self, ppml, layout: SlabLayout, h, gamma, cfl, dtype, u_padded, rho_ref,
                 vacuum_frac=1e-5, t_end=0.0, device="cuda"):
        self.ppml, self.L = ppml, layout
        self.cur = u_padded
        self.nxt = [alloc_padded(layout, x.dtype, x.device) for x in u_padded]
        self.star = [alloc_padded(layout, x.dtype, x.device) for x in u_padded]
        self.red = torch.zeros(REDUCE_LEN, dtype=torch.float64, device=device)
        self.grid = ppml.Grid(layout.slab_n, h, gamma, cfl, layout.slab_bc, dtype,
                              u0=self.state(self.cur), vacuum_frac=vacuum_frac, t_end=t_end,
                              rho_ref=rho_ref)

    def state(self, fields):
        st = self.ppml.State()
        off = self.L.pad_lo * self.L.plane * fields[0].element_size()
        for f, t in enumerate(fields):
            st.f[f] = t.data_ptr() + off
        return st

    def star_state(self):
        """U*: the Eulerian stage leaves rho unchanged, so U*'s rho is U^n's array (its
        halo planes come with U^n's exchange)."""
        st = self.state(self.star)
        st.f[0] = self.state(self.cur).f[0]
        return st

    def local_reduce(self):
        self.grid.local_reduce(self.state(self.cur), self.red)

    def eulerian(self, dt):
        self.grid.eulerian_stage_ptrs(self.state(self.cur), self.star_state(), dt)

    def lagrangian(self, dt):
        self.grid.lagrangian_stage(self.star_state(), self.state(self.nxt), dt, self.red)

    def apply(self, advance, dt):
        self.grid.apply_reduced(self.red, advance, dt)
        if advance:
            self.cur, self.nxt = self.nxt, self.cur

    @property
    def star_fields(self):
        """The U* arrays exchanged between the stages (m, rho E, rho eps; rho is U^n's)."""
        return self.star[1:]


def start(stages, comm):
    """The first CFL step of the decomposed grid: each slab's maxima, all-reduced."""
    for s in stages:
        s.local_reduce()
    _reduce(stages, comm)
    for s in stages:
        s.apply(False, 0.0)


def step(stages, comm, dt=0.0):
    """One step of every slab (the slabs of this process: one per rank with DistComm, all
    of them with LocalComm).  dt > 0: that step size; dt <= 0: the device-resident CFL step
    each slab holds (equal on all slabs after the all-reduce)."""
    _exchange(stages, comm, "cur")
    for s in stages:
        s.eulerian(dt)
    _exchange(stages, comm, "star_fields")
    for s in stages:
        s.lagrangian(dt)
    _reduce(stages, comm)
    for s in stages:
        s.apply(True, dt)


def _exchange(stages, comm, which):
    if isinstance(comm, LocalComm):
        comm.exchange([getattr(s, which) for s in stages])
    else:
        for s in stages:
            comm.exchange(getattr(s, which))


def _reduce(stages, comm):
    if isinstance(comm, LocalComm):
        comm.allreduce([s.red for s in stages])
    else:
        for s in stages:
            comm.allreduce(s.red)


def alloc_padded(layout: SlabLayout, dtype, device):
    """A zeroed halo-padded field whose first interior plane starts on a 16-byte boundary
    (the library's alignment rule for state pointers): a view behind a short lead."""
    elt = torch.empty((), dtype=dtype).element_size()
    lead = (-(layout.pad_lo * layout.plane)) % (16 // elt)
    n = layout.planes * layout.plane
    return torch.zeros(lead + n, dtype=dtype, device=device)[lead:]


def pad_field(layout: SlabLayout, whole, dtype, device):
    """The slab's planes of a whole-grid field (flat, x fastest) in a halo-padded tensor; the
    halo planes are filled by the first exchange."""
    t = alloc_padded(layout, dtype, device)
    src = torch.as_tensor(whole).reshape(-1)[layout.z0 * layout.plane:(layout.z0 + layout.nz) * layout.plane]
    layout.interior(t).copy_(src.to(device=device, dtype=dtype))
    return t
