"""Inflow boundaries (PPML_BC_INFLOW) on the GPU against the FP64 oracle, through the C ABI.

An inflow face's ghost cells hold a prescribed conserved state; at an edge or corner of two
ghost regions the later axis (x, y, z order of the ghost fill) decides.  The FP64 kernels
must reproduce the oracle bit for bit on boundary tiles, ragged tiles, edges where two
inflow faces meet, the 2D and 1D modes and interior tiles; FP32 within the single-step bar.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_1607_01105_gb300 import inputs, ppml  # noqa: E402

pytestmark = pytest.mark.gpu

F32, F64 = ppml.PPML_F32, ppml.PPML_F64
IN = ppml.INFLOW
GAMMA = 1.4


def _state(rho, mx, my, mz, p):
    ei = p / (GAMMA - 1.0)
    return (rho, mx, my, mz, ei + 0.5 * (mx * mx + my * my + mz * mz) / rho, ei)


# one prescribed state per face, all different (and different from the interiors)
STATES = {0: _state(1.3, 0.4, -0.2, 0.1, 1.1), 1: _state(0.8, -0.3, 0.05, 0.0, 0.9),
          2: _state(1.1, 0.0, 0.3, -0.1, 1.2), 3: _state(0.7, 0.1, -0.25, 0.05, 1.4),
          4: _state(0.9, 0.1, 0.1, 0.35, 1.0), 5: _state(1.2, -0.1, 0.0, -0.25, 0.8)}

CASES = {
    # x-lo and z-hi inflow (their edge: z decides), periodic y, an interior tile
    "inflow_3d": lambda: inputs.random_rough(n=(37, 35, 36), bc=(IN, 0, 1, 1, 0, IN)),
    # ragged tiles, inflow on both x faces and on z-lo
    "inflow_ragged_3d": lambda: inputs.random_rough(n=(19, 13, 11), bc=(IN, IN, 0, 0, IN, 0)),
    "inflow_2d": lambda: inputs.random_rough(n=(37, 29, 1), bc=(IN, 0, 0, IN, 0, 0)),
    "inflow_1d": lambda: inputs.random_rough(n=(301, 1, 1), bc=(0, IN, 0, 0, 0, 0)),
}


def _inflow(pb):
    return {q: STATES[q] for q in range(6) if pb.bc[q] == IN}


def _oracle_grid(pb):
    return oracle.Grid(pb.n, pb.h, pb.gamma, pb.bc, pb.cfl, rho_mean=oracle.mean_density(pb.u),
                       inflow=_inflow(pb))


def _gpu_grid(pb, dtype, u):
    return ppml.Grid(pb.n, pb.h, pb.gamma, pb.cfl, pb.bc, dtype, u0=u, inflow=_inflow(pb))


def _host(u, pb):
    return [t.double().cpu().numpy().reshape(pb.n[2], pb.n[1], pb.n[0]) for t in u]


def _rel_l1(got, ref, scale=None):
    den = np.abs(ref).sum()
    if scale is not None:
        den = max(den, 1e-3 * np.abs(scale).sum())
    return float(np.abs(got - ref).sum() / den)


@pytest.mark.parametrize("case", sorted(CASES))
def test_inflow_fp64_bitwise_equal_to_oracle(case):
    """One step and its Eulerian stage bit for bit; three steps with the device CFL step."""
    pb = CASES[case]()
    assert pb.gamma == GAMMA
    g = _oracle_grid(pb)
    dt = oracle.cfl_dt(g, pb.u)
    ref, _, ustar = oracle.step(g, pb.u, dt, want_star=True)
    u = ppml.to_device(pb.u, F64)
    v = [torch.empty_like(x) for x in u]
    s = [torch.empty_like(x) for x in u]
    grid = _gpu_grid(pb, F64, u)
    grid.eulerian_stage(u, s, dt)
    grid.step(u, v, dt)
    got_s, got = _host(s, pb), _host(v, pb)
    assert [int(np.count_nonzero(got_s[f] != ustar[f])) for f in range(6)] == [0] * 6
    assert [int(np.count_nonzero(got[f] != ref[f])) for f in range(6)] == [0] * 6
    # three steps with the device-resident CFL step
    u = ppml.to_device(pb.u, F64)
    grid = _gpu_grid(pb, F64, u)
    ref = pb.u
    for _ in range(3):
        ref, dg = oracle.step(g, ref, oracle.cfl_dt(g, ref))
        grid.step(u, v, 0.0)
        u, v = v, u
    got = _host(u, pb)
    assert [int(np.count_nonzero(got[f] != ref[f])) for f in range(6)] == [0] * 6
    assert grid.diag()["dt_next"] == pytest.approx(dg["dt_cfl"], rel=1e-12)


@pytest.mark.parametrize("case", ["inflow_3d", "inflow_2d"])
def test_inflow_fp32_single_step(case):
    """One FP32 step from the same (float-representable) input: rho and p within 1e-5."""
    pb = CASES[case]()
    pb.u = [a.astype(np.float32).astype(np.float64) for a in pb.u]
    g = _oracle_grid(pb)
    dt = oracle.cfl_dt(g, pb.u)
    ref, _ = oracle.step(g, pb.u, dt)
    u = ppml.to_device(pb.u, F32)
    v = [torch.empty_like(x) for x in u]
    grid = _gpu_grid(pb, F32, u)
    grid.step(u, v, dt)
    got = _host(v, pb)
    assert _rel_l1(got[0], ref[0]) <= 1e-5
    assert _rel_l1(got[5], ref[5]) <= 1e-5


def test_inflow_supersonic_riemann_run_fp64():
    """The oracle's inflow pin on the GPU: gas at rest on [0, 1] with a supersonic inflow
    (rho = 1, u = 3, p = 1) at x = 0, 200 cells, run to t = 0.3 with the device CFL step:
    the same 702 steps and the same state as the oracle, within 1e-12."""
    n = 200
    z = np.zeros(n)
    u0 = [a[None, None, :] for a in (np.ones(n), z, z, z, np.full(n, 2.5), np.full(n, 2.5))]
    bc = (IN, 0, 0, 0, 0, 0)
    inflow = {0: (1.0, 3.0, 0.0, 0.0, 7.0, 2.5)}
    g = oracle.Grid((n, 1, 1), (1.0 / n, 1.0, 1.0), GAMMA, bc, 0.4, rho_mean=1.0, inflow=inflow)
    ref, t, steps, _ = oracle.run(g, u0, 0.3)
    u = ppml.to_device(u0, F64)
    v = [torch.empty_like(x) for x in u]
    grid = ppml.Grid((n, 1, 1), (1.0 / n, 1.0, 1.0), GAMMA, 0.4, bc, F64, u0=u, t_end=0.3,
                     inflow=inflow)
    k = 0
    while grid.diag()["t"] < 0.3 and k < 2 * steps:
        grid.step(u, v, 0.0)
        u, v = v, u
        k += 1
    d = grid.diag()
    assert d["steps"] == steps and d["t"] == pytest.approx(t, rel=1e-14)
    got = [x.cpu().numpy().reshape(1, 1, n) for x in u]
    for f in (0, 1, 4, 5):
        assert _rel_l1(got[f], ref[f]) <= 1e-12, f


def test_inflow_faces_refused_without_a_handle():
    pb = CASES["inflow_1d"]()
    u = ppml.to_device(pb.u, F64)
    v = [torch.empty_like(x) for x in u]
    d = ppml.make_desc(pb.n, pb.h, pb.gamma, pb.cfl, pb.bc, F64)
    with pytest.raises(ppml.PPMLError):
        ppml.step_noalloc(d, u, v, 1e-4, 1.0)
    with pytest.raises(ValueError):  # an inflow face needs its state
        ppml.Grid(pb.n, pb.h, pb.gamma, pb.cfl, pb.bc, F64, u0=u)
