"""z-slab decomposition of the step (paper_1607_01105_gb300/slab.py) on CPU gloo ranks.

Each rank holds a slab of the grid's z planes with halo planes behind its shared faces and
runs the decomposition exactly as on GPUs -- layout, the exchange of U^n and U* halo
planes, the all-reduce of the CFL maxima and sums, the order of the step -- with the two
stages computed by the FP64 oracle on the halo-extended slab instead of the kernels (the
test harness below; no GPU here).  The assembled state must equal the single-grid oracle
run bit for bit: every cell takes the same operations on the same values, and the CFL
step comes from the same maxima.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
from paper_1607_01105_gb300 import inputs, slab  # noqa: E402


class OracleStages:
    """The calls of slab.Stages computed by the FP64 oracle on the host: the Eulerian stage
    and the second half of the step on the slab extended by its halo planes (the halo
    planes' own results, which depend on cells beyond them, are discarded)."""

    def __init__(self, layout, pb, rho_ref):
        self.L, self.pb = layout, pb
        self.cur = [slab.pad_field(layout, u, torch.float64, "cpu") for u in pb.u]
        self.nxt = [slab.alloc_padded(layout, torch.float64, "cpu") for _ in range(6)]
        self.star = [slab.alloc_padded(layout, torch.float64, "cpu") for _ in range(6)]
        self.red = torch.zeros(slab.REDUCE_LEN, dtype=torch.float64)
        nx, ny, nz = layout.slab_n
        bc = tuple(slab.OUTFLOW if b == slab.HALO else b for b in layout.slab_bc)
        self.g_ext = oracle.Grid((nx, ny, layout.planes), pb.h, pb.gamma, bc, pb.cfl, rho_mean=rho_ref)
        self.g_int = oracle.Grid(layout.slab_n, pb.h, pb.gamma, bc, pb.cfl, rho_mean=rho_ref)
        self.hmin = min(pb.h[a] for a in range(3) if pb.n[a] > 1)
        self.dt = 0.0

    def _ext(self, fields):
        L = self.L
        return [t.numpy().reshape(L.planes, L.n[1], L.n[0]) for t in fields]

    def _interior(self, arrs):
        L = self.L
        return [a[L.pad_lo:L.pad_lo + L.nz] for a in arrs]

    def _put(self, dst, arrs):
        for t, a in zip(dst, self._interior(arrs)):
            self.L.interior(t).copy_(torch.from_numpy(np.ascontiguousarray(a).reshape(-1)))

    def _reduce_of(self, fields):
        dg = oracle.diagnostics(self.g_int, self._interior(self._ext(fields)))
        self.red.copy_(torch.tensor([dg["vmax"], dg["cmax"]] + list(dg["sums"]) +
                                    [0.0, float(dg["n_nonphys"])], dtype=torch.float64))

    def local_reduce(self):
        self._reduce_of(self.cur)

    def eulerian(self, dt):
        tau = dt if dt > 0 else self.dt
        _, _, star = oracle.step(self.g_ext, self._ext(self.cur), tau, want_star=True)
        self._put(self.star, star)

    def lagrangian(self, dt):
        tau = dt if dt > 0 else self.dt
        out, _ = oracle.lagrangian_step(self.g_ext, self._ext(self._star_with_rho()), tau)
        self._put(self.nxt, out)
        self._reduce_of(self.nxt)

    def apply(self, advance, dt):
        self.dt = self.pb.cfl * self.hmin / (float(self.red[0]) + float(self.red[1]))
        if advance:
            self.cur, self.nxt = self.nxt, self.cur

    @property
    def star_fields(self):  # as slab.Stages: rho of U* is U^n's, exchanged with U^n
        return self.star[1:]

    def _star_with_rho(self):
        return [self.cur[0]] + self.star[1:]


def _case(name):
    if name == "periodic_z":
        pb = inputs.random_rough(n=(8, 8, 12), bc=(0, 0, 1, 1, 1, 1))
    else:  # reflecting bottom, outflow top, periodic x
        pb = inputs.random_rough(n=(8, 4, 13), bc=(1, 1, 0, 0, 2, 0))
    return pb


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, name, steps, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pb = _case(name)
    L = slab.SlabLayout(pb.n, pb.bc, world, rank)
    st = OracleStages(L, pb, oracle.mean_density(pb.u))
    comm = slab.DistComm(dist, L)
    slab.start([st], comm)
    dts = []
    for _ in range(steps):
        dts.append(st.dt)
        slab.step([st], comm, 0.0)
    out.put((rank, L.z0, L.nz, [L.interior(t).numpy().copy() for t in st.cur], dts))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("name,world", [("periodic_z", 2), ("walls_z", 3)])
def test_slab_decomposition_equals_single_grid(name, world):
    steps = 3
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, name, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = sorted(q.get() for _ in range(world))
    pb = _case(name)
    g = oracle.Grid(pb.n, pb.h, pb.gamma, pb.bc, pb.cfl, rho_mean=oracle.mean_density(pb.u))
    u, dt, dts = pb.u, oracle.cfl_dt(g, pb.u), []
    for _ in range(steps):
        dts.append(dt)
        u, dg = oracle.step(g, u, dt)
        dt = dg["dt_cfl"]
    plane = pb.n[0] * pb.n[1]
    for rank, z0, nz, fields, rank_dts in res:
        assert rank_dts == dts  # the same CFL steps, bit for bit
        for f in range(6):
            ref = u[f].reshape(-1)[z0 * plane:(z0 + nz) * plane]
            assert np.array_equal(fields[f], ref), (rank, f)


def test_slab_layout():
    """Slab sizes cover the grid; halo faces only where slabs meet (and on both faces of
    every slab of a periodic z axis); too thin slabs are refused."""
    for nz, world in ((12, 2), (13, 3), (256, 8)):
        Ls = [slab.SlabLayout((8, 8, nz), (0, 0, 0, 0, 2, 0), world, r) for r in range(world)]
        assert sum(L.nz for L in Ls) == nz and Ls[0].z0 == 0
        assert all(a.z0 + a.nz == b.z0 for a, b in zip(Ls, Ls[1:]))
        assert Ls[0].slab_bc[4] == 2 and Ls[-1].slab_bc[5] == 0
        assert all(L.slab_bc[4] == slab.HALO for L in Ls[1:])
        assert all(L.slab_bc[5] == slab.HALO for L in Ls[:-1])
    P = [slab.SlabLayout((8, 8, 12), (0, 0, 0, 0, 1, 1), 2, r) for r in range(2)]
    assert all(L.slab_bc[4:] == (slab.HALO, slab.HALO) for L in P)
    single = slab.SlabLayout((8, 8, 12), (0, 0, 0, 0, 1, 1), 1, 0)
    assert single.slab_bc[4:] == (1, 1) and single.planes == 12
    # boundaries on 16-plane tiles where that keeps every slab at >= 3 planes
    assert slab.slab_bounds(36, 2) == [0, 16, 36] and slab.slab_bounds(45, 3) == [0, 16, 32, 45]
    assert slab.slab_bounds(256, 8) == list(range(0, 257, 32))
    assert slab.slab_bounds(12, 2) == [0, 6, 12] and slab.slab_bounds(13, 3) == [0, 5, 9, 13]
    with pytest.raises(ValueError):
        slab.SlabLayout((8, 8, 5), (0,) * 6, 2, 1)  # planes 3 + 2
