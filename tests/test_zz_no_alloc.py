"""ppml_step_noalloc: the step for callers that cannot call cudaMalloc (code running
while a CUDA graph is being captured elsewhere in the process, plugins inside a host
application that owns the device memory, real-time loops).  It must give the same
result as the handle-based ppml_step, call after call, although it keeps its scratch in
one fixed buffer of the library instead of allocating.  This file sorts last so that a
run stopping at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1607_01105_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1607_01105_gb300 import ppml  # noqa: E402


@pytest.mark.parametrize("dtype,n", [(ppml.PPML_F64, (40, 24, 20)), (ppml.PPML_F32, (40, 24, 20)),
                                     (ppml.PPML_F64, (64, 64, 64)), (ppml.PPML_F64, (17, 17, 907))])
def test_noalloc_step_matches_handle_step_twice(dtype, n):
    """Two calls in a row against the handle-based step, on a small grid, on a grid of
    exactly the buffer's limit (64^3 = PPML_NOALLOC_MAX_CELLS cells) and on a thin grid
    with ragged tiles (17 x 17 x 907 = 262123 cells, 228 tiles)."""
    assert n[0] * n[1] * n[2] <= ppml.NOALLOC_MAX_CELLS
    pb = inputs.random_smooth(n=n, bc=(0, 0, 1, 1, 0, 0))
    rho_mean = oracle.mean_density(pb.u)
    u0 = ppml.to_device(pb.u, dtype)
    grid = ppml.Grid(pb.n, pb.h, pb.gamma, pb.cfl, pb.bc, dtype, u0=u0)
    desc = ppml.make_desc(pb.n, pb.h, pb.gamma, pb.cfl, pb.bc, dtype)
    dt = 0.8 * grid.cfl_dt(u0)
    ref = [x.clone() for x in u0]
    got = [x.clone() for x in u0]
    tmp_ref = [torch.empty_like(x) for x in u0]
    tmp_got = [torch.empty_like(x) for x in u0]
    for call in range(2):  # two calls in a row share the fixed buffer
        grid.step(ref, tmp_ref, dt)
        diag = ppml.step_noalloc(desc, got, tmp_got, dt, rho_mean)
        torch.cuda.synchronize()
        ref, tmp_ref = tmp_ref, ref
        got, tmp_got = tmp_got, got
        d = grid.diag()
        for f in range(6):
            a = got[f].double().cpu().numpy()
            b = ref[f].double().cpu().numpy()
            scale = max(np.abs(b).sum(), np.abs(ref[0].double().cpu().numpy()).sum())
            assert np.abs(a - b).sum() <= 1e-10 * scale, (call, f)
        assert diag[0] == pytest.approx(d["dt_next"], rel=1e-10)
        for f in range(6):
            assert diag[3][f] == pytest.approx(d["sums"][f], rel=1e-10, abs=1e-10 * abs(d["sums"][0]))


def test_noalloc_rejects_grids_beyond_its_buffer():
    n = (80, 80, 80)  # 512000 cells > PPML_NOALLOC_MAX_CELLS
    assert n[0] * n[1] * n[2] > ppml.NOALLOC_MAX_CELLS
    desc = ppml.make_desc(n, (0.01,) * 3, 1.4, 0.2)
    dummy = [torch.empty(16, device="cuda") for _ in range(6)]
    st = ppml.State()
    for i, t in enumerate(dummy):
        st.f[i] = t.data_ptr()
    out = (ctypes.c_double * 9)()
    rc = ppml.lib().ppml_step_noalloc(ctypes.byref(desc), ctypes.byref(st), ctypes.byref(st), 1e-3,
                                      1.0, out, None)
    assert rc == ppml.PPML_E_INVAL
    assert "fixed buffer" in ppml.lib().ppml_last_error().decode()


def test_noalloc_rejects_end_time_and_low_parts():
    """The call keeps no simulated time (t_end must be 0) and takes plain states only."""
    pb = inputs.random_smooth(n=(16, 8, 8))
    u = ppml.to_device(pb.u, ppml.PPML_F32)
    v = [torch.empty_like(x) for x in u]
    desc = ppml.make_desc(pb.n, pb.h, pb.gamma, pb.cfl, pb.bc, ppml.PPML_F32, t_end=0.5)
    with pytest.raises(ppml.PPMLError) as e:
        ppml.step_noalloc(desc, u, v, 1e-4, 1.0)
    assert e.value.code == ppml.PPML_E_INVAL and "t_end" in str(e.value)
    desc = ppml.make_desc(pb.n, pb.h, pb.gamma, pb.cfl, pb.bc, ppml.PPML_F32)
    ud = ppml.to_device(pb.u, ppml.PPML_F32, lo=True)
    vd = [torch.empty_like(x) for x in ud]
    with pytest.raises(ppml.PPMLError) as e:
        ppml.step_noalloc(desc, ud, vd, 1e-4, 1.0)
    assert e.value.code == ppml.PPML_E_INVAL
