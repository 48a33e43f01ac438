"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every
function include/ppml.h declares, and rejects invalid arguments before touching CUDA."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ppml.h")
LIB = os.path.join(ROOT, "paper_1607_01105_gb300", "libppml.so")


@pytest.fixture(scope="module")
def built():
    if not os.path.exists(LIB):
        import __graft_entry__
        __graft_entry__.build()
    return LIB


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_]+\**\s+\**(ppml_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ppml_init_grid", "ppml_step", "ppml_cfl_dt", "ppml_batch_step",
                     "ppml_free_grid", "ppml_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_matches_header(built):
    from paper_1607_01105_gb300 import ppml
    assert sorted(ppml.EXPORTED) == declared_functions()


def test_invalid_descriptors_rejected_on_host(built):
    from paper_1607_01105_gb300 import ppml
    lib = ppml.lib()

    def init(**kw):
        d = ppml.GridDesc()
        d.nx, d.ny, d.nz = kw.get("n", (8, 8, 8))
        for a in range(3):
            d.h[a] = kw.get("h", 0.1)
        d.gamma = kw.get("gamma", 1.4)
        d.cfl = kw.get("cfl", 0.2)
        for q, v in enumerate(kw.get("bc", (0,) * 6)):
            d.bc[q] = v
        d.dtype = kw.get("dtype", 0)
        for q, state in kw.get("inflow", {}).items():
            for f in range(6):
                d.inflow[q][f] = state[f]
        h = ctypes.c_void_p()
        rc = lib.ppml_init_grid(ctypes.byref(d), None, None, ctypes.byref(h))
        return rc, lib.ppml_last_error().decode()

    assert init(gamma=1.0)[0] == ppml.PPML_E_INVAL
    assert init(cfl=1.5)[0] == ppml.PPML_E_INVAL
    assert init(n=(0, 4, 4))[0] == ppml.PPML_E_INVAL
    assert init(n=(2, 4, 4))[0] == ppml.PPML_E_INVAL
    assert init(h=-1.0)[0] == ppml.PPML_E_INVAL
    assert init(bc=(1, 0, 0, 0, 0, 0))[0] == ppml.PPML_E_INVAL  # unpaired periodic
    assert init(n=(8, 1, 1), bc=(0, 0, 2, 2, 0, 0))[0] == ppml.PPML_E_INVAL
    assert init(dtype=7)[0] == ppml.PPML_E_INVAL
    assert init(bc=(5, 0, 0, 0, 0, 0))[0] == ppml.PPML_E_INVAL
    good = {0: (1.0, 3.0, 0.0, 0.0, 7.0, 2.5)}
    assert init(bc=(ppml.INFLOW,) + (0,) * 5, inflow={0: (0.0,) * 6})[0] == ppml.PPML_E_INVAL
    rc, msg = init(bc=(ppml.INFLOW, 0, 2, 2, 0, 0), inflow=good)  # inflow with a wall
    assert rc == ppml.PPML_E_INVAL and "reflecting" in msg
    rc, msg = init(bc=(ppml.INFLOW,) + (0,) * 5, inflow=good)  # valid, but no initial state
    assert rc == ppml.PPML_E_INVAL and "u0" in msg
    rc, msg = init()  # valid descriptor but no initial state
    assert rc == ppml.PPML_E_INVAL and "u0" in msg
    # batch validation
    h = ctypes.c_void_p()
    nc = (ctypes.c_int * 2)(64, 2)
    hh = (ctypes.c_double * 2)(0.1, 0.1)
    te = (ctypes.c_double * 2)(0.1, 0.1)
    assert lib.ppml_batch_init(2, nc, hh, te, 1.4, 0.4, 0.0, 0, ctypes.byref(h)) == ppml.PPML_E_INVAL
    assert lib.ppml_batch_init(2, nc, hh, te, 1.4, 1.4, 0.0, 0, ctypes.byref(h)) == ppml.PPML_E_INVAL
    assert lib.ppml_step(None, None, None, ctypes.c_double(0.1), None) == ppml.PPML_E_INVAL
    assert lib.ppml_free_grid(None) == ppml.PPML_OK
    assert lib.ppml_poisson_isolated(None, None, None, 1.0, 0, None) == ppml.PPML_E_INVAL
    assert lib.ppml_poisson_periodic(None, None, None, 1.0, None) == ppml.PPML_E_INVAL


def test_batch_work_plan_on_host(built):
    """The batch work plan (host logic, no device call): every instance appears exactly once;
    instances of at least split_min cells, and only they, are split over a CTA pair; the
    items come largest first by their largest instance, whole instances paired in order of
    size; with no split the plan is one CTA per instance, largest first (stable).  Invalid
    thresholds are rejected."""
    import numpy as np
    from paper_1607_01105_gb300 import ppml
    rng = np.random.default_rng(5)
    cells = [int(x) for x in 2 * rng.integers(64, 2049, size=101)]
    for split_min in (1024, 2000, 3000, 64):
        items, order = ppml.batch_plan(cells, split_min)
        assert order is None and items
        seen = []
        for a, b in items:
            seen.append(a)
            if b == -2:
                assert cells[a] >= split_min
            else:
                assert cells[a] < split_min
                if b >= 0:
                    assert cells[b] < split_min and cells[b] <= cells[a]
                    seen.append(b)
        assert sorted(seen) == list(range(len(cells)))
        keys = [cells[a] for a, _ in items]
        assert keys == sorted(keys, reverse=True)
        whole = [x for a, b in items if b != -2 for x in (a, b) if x >= 0]
        assert [cells[x] for x in whole] == sorted((cells[x] for x in whole), reverse=True)
        assert sum(1 for _, b in items if b == -1) <= 1
    items, order = ppml.batch_plan(cells, 10 ** 6)  # nothing large enough: one CTA each
    assert items == [] and order == sorted(range(len(cells)), key=lambda i: (-cells[i], i))
    items, order = ppml.batch_plan(cells, 0)
    assert items == [] and order == sorted(range(len(cells)), key=lambda i: (-cells[i], i))
    for bad in (10, -1):
        with pytest.raises(ppml.PPMLError):
            ppml.batch_plan(cells, bad)
