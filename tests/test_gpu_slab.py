"""z-slab decomposition on the GPU: several slabs of one grid driven by one process (halo
planes copied between the slabs' arrays, the ten reduced scalars combined in rank order),
through the library's slab calls, against the single-grid ppml_step.  Every cell takes the
same operations on the same values, so the states agree bit for bit in FP64 and FP32."""
import numpy as np
import pytest

import oracle
from paper_1607_01105_gb300 import inputs, slab

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU, skipped there
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1607_01105_gb300 import ppml  # noqa: E402


def _slabs(pb, dtype, world):
    Ls = [slab.SlabLayout(pb.n, pb.bc, world, r) for r in range(world)]
    td = ppml.torch_dtype(dtype)
    rho_ref = oracle.mean_density(pb.u)
    st = [slab.Stages(ppml, L, pb.h, pb.gamma, pb.cfl, dtype,
                      [slab.pad_field(L, u, td, "cuda") for u in pb.u], rho_ref) for L in Ls]
    return Ls, st


@pytest.mark.parametrize("dtype", [ppml.PPML_F64, ppml.PPML_F32])
@pytest.mark.parametrize("case,world", [("periodic", 2), ("walls", 3), ("blast", 2)])
def test_slabs_equal_single_grid(case, world, dtype):
    pb = {"periodic": lambda: inputs.random_rough(n=(40, 20, 36), bc=(0, 0, 1, 1, 1, 1)),
          "walls": lambda: inputs.random_smooth(n=(24, 16, 45), bc=(2, 0, 1, 1, 2, 0)),
          "blast": lambda: inputs.point_blast_3d(64)}[case]()
    steps = 4
    u = ppml.to_device(pb.u, dtype)
    v = [torch.empty_like(x) for x in u]
    grid = ppml.Grid(pb.n, pb.h, pb.gamma, pb.cfl, pb.bc, dtype, u0=u)
    for _ in range(steps):
        grid.step(u, v, 0.0)
        u, v = v, u
    ref = [x.reshape(pb.n[2], -1) for x in u]
    d = grid.diag()
    Ls, st = _slabs(pb, dtype, world)
    comm = slab.LocalComm(Ls)
    slab.start(st, comm)
    for _ in range(steps):
        slab.step(st, comm, 0.0)
    for L, s in zip(Ls, st):
        ds = s.grid.diag()
        assert ds["dt_next"] == d["dt_next"] and ds["t"] == d["t"] and ds["steps"] == steps
        assert ds["vmax"] == d["vmax"] and ds["cmax"] == d["cmax"]
        for f in range(6):
            got = L.interior(s.cur[f]).reshape(L.nz, -1)
            assert torch.equal(got, ref[f][L.z0:L.z0 + L.nz]), (L.rank, f)
        for f in range(6):  # the same sums, added in another order
            assert ds["sums"][f] == pytest.approx(d["sums"][f], rel=1e-12, abs=1e-12 * abs(d["sums"][0]))


def test_halo_grids_refused_by_calls_without_halo_planes():
    """ppml_step, ppml_step_phi, the Poisson solves and the tuner step through the handle's
    own U*, which has no halo planes: they refuse grids with halo faces."""
    pb = inputs.random_smooth(n=(16, 8, 12), bc=(0, 0, 1, 1, 1, 1))
    Ls, st = _slabs(pb, ppml.PPML_F64, 2)
    s = st[0]
    out = s.state(s.nxt)
    rc = ppml.lib().ppml_step(s.grid._h, s.state(s.cur), out, 1e-4, None)
    assert rc == ppml.PPML_E_INVAL and "halo" in ppml.lib().ppml_last_error().decode()
    phi = torch.zeros(Ls[0].cells, dtype=torch.float64, device="cuda")
    rc = ppml.lib().ppml_step_phi(s.grid._h, s.state(s.cur), out, phi.data_ptr(), 1e-4, None)
    assert rc == ppml.PPML_E_INVAL
    with pytest.raises(ppml.PPMLError):
        s.grid.poisson_periodic(phi, torch.empty_like(phi))
    with pytest.raises(ppml.PPMLError):
        s.grid.poisson_isolated(phi, torch.empty_like(phi))
    rc = ppml.lib().ppml_grid_tune(s.grid._h, s.state(s.cur), 1, None, None, None)
    assert rc == ppml.PPML_E_INVAL
    with pytest.raises(ppml.PPMLError):  # halo faces are z faces only
        ppml.Grid((16, 8, 12), pb.h, pb.gamma, pb.cfl, (3, 0, 1, 1, 1, 1), ppml.PPML_F64,
                  u0=ppml.to_device(pb.u, ppml.PPML_F64))
