"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms,
textbook special cases, exact solutions, invariants, values the paper prints
(tests/golden/paper_values.json) and brute force on small inputs.  A dropped term,
a wrong sign, a swapped index or a transposed operand anywhere in the scheme fails at
least one of them (see the per-test docstrings).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import exact
from paper_1607_01105_gb300 import inputs

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def grid_of(pb, **kw):
    return oracle.Grid(pb.n, pb.h, pb.gamma, pb.bc, pb.cfl,
                       rho_mean=oracle.mean_density(pb.u), **kw)


def parabola_eval(qL, dq, q6, xi):
    """Eq. A1 of the Appendix: q(xi) = qL + xi (dq + q6 (1 - xi))."""
    return qL + xi * (dq + q6 * (1.0 - xi))


def quad(fn, a, b, n=8):
    x, w = np.polynomial.legendre.leggauss(n)
    xs = 0.5 * (a + b) + 0.5 * (b - a) * x
    return 0.5 * (b - a) * np.sum(w * fn(xs))


# ------------------------------------------------------------------ parabolas (S1)

def test_golden_inputs_match_table2():
    """The generators use the shock-tube states printed in Table 2."""
    for row, vals in GOLDEN["shock_tubes"]["rows"].items():
        assert tuple(float(v) for v in vals) == inputs.SOD_TABLE2[int(row)]


def test_parabola_constant_is_flat():
    qL, qR, dq, q6 = oracle.line_parabolas(np.full(12, 3.25))
    c = slice(2, 10)
    assert np.all(qL[c] == 3.25) and np.all(qR[c] == 3.25)
    assert np.all(dq[c] == 0.0) and np.all(q6[c] == 0.0)


def test_parabola_linear_exact():
    """Linear data: faces at the exact point values, q6 = 0, averages exact."""
    i = np.arange(16, dtype=np.float64)
    q = 2.0 + 0.75 * i
    qL, qR, dq, q6 = oracle.line_parabolas(q)
    for c in range(2, 14):
        assert qL[c] == pytest.approx(2.0 + 0.75 * (c - 0.5), abs=1e-14)
        assert qR[c] == pytest.approx(2.0 + 0.75 * (c + 0.5), abs=1e-14)
        assert abs(q6[c]) < 1e-13
        y = 0.3
        # mean of the linear function over the right fraction y of cell c
        exact_r = 2.0 + 0.75 * (c + 0.5 - 0.5 * y)
        exact_l = 2.0 + 0.75 * (c - 0.5 + 0.5 * y)
        assert oracle.avg_right_part(qR[c], dq[c], q6[c], y) == pytest.approx(exact_r, abs=1e-13)
        assert oracle.avg_left_part(qL[c], dq[c], q6[c], y) == pytest.approx(exact_l, abs=1e-13)


def test_face_interpolant_exact_for_cubics():
    """Appendix: the 4th-order face formula from cell averages reproduces a cubic's point
    values at the faces (unlimited slopes on monotone data).  Catches a wrong 1/2 or 1/6
    coefficient, a swapped delta index or a sign error in the face formula."""
    h = 0.05
    poly = np.polynomial.Polynomial([0.3, 1.0, 0.4, 0.2])  # increasing on [0, 1]
    P = poly.integ()
    edges = np.arange(21) * h
    q = (P(edges[1:]) - P(edges[:-1])) / h
    qL, qR, dq, q6 = oracle.line_parabolas(q)
    for c in range(3, 17):
        assert qR[c] == pytest.approx(poly(edges[c + 1]), abs=1e-12)
        assert qL[c] == pytest.approx(poly(edges[c]), abs=1e-12)


def test_parabola_conserves_cell_average_random():
    """Appendix (integral property below eq. A1): the mean of every final parabola over
    its cell equals the cell value.  Checked by quadrature of eq. A1 with the returned
    coefficients; a wrong q6 or Delta q (e.g. the printed qL - qR sign) fails it."""
    rng = np.random.default_rng(11)
    for _ in range(50):
        q = rng.normal(size=40) * rng.uniform(0.1, 10)
        qL, qR, dq, q6 = oracle.line_parabolas(q)
        for c in range(2, 38):
            m = quad(lambda x: parabola_eval(qL[c], dq[c], q6[c], x), 0.0, 1.0, 4)
            assert m == pytest.approx(q[c], rel=1e-12, abs=1e-12)
            assert qR[c] == pytest.approx(parabola_eval(qL[c], dq[c], q6[c], 1.0), abs=1e-12)


def test_parabola_monotone_no_new_extrema():
    """Appendix Step 2: after the monotonicity fixes each parabola is monotone on its cell
    and stays within the range of the cell and its two neighbours (brute-force scan)."""
    rng = np.random.default_rng(12)
    xi = np.linspace(0.0, 1.0, 201)
    for trial in range(200):
        q = rng.normal(size=24)
        if trial % 3 == 0:
            q = np.cumsum(np.abs(q))  # monotone data with kinks
        qL, qR, dq, q6 = oracle.line_parabolas(q)
        for c in range(2, 22):
            vals = parabola_eval(qL[c], dq[c], q6[c], xi)
            d = np.diff(vals)
            tol = 1e-12 * (1.0 + np.max(np.abs(vals)))
            assert np.all(d >= -tol) or np.all(d <= tol)
            lo = min(q[c - 1], q[c], q[c + 1]) - tol
            hi = max(q[c - 1], q[c], q[c + 1]) + tol
            assert vals.min() >= lo and vals.max() <= hi


def test_characteristic_averages_match_quadrature():
    """Appendix, characteristic integrals: q_L(-lambda t) and q_R(lambda t) are the means
    of eq. A1 over the right / left fraction y of the cell (independent quadrature)."""
    rng = np.random.default_rng(13)
    for _ in range(200):
        qL, dq, q6 = rng.normal(size=3)
        y = rng.uniform(0.0, 1.0)
        qR = qL + dq
        right = quad(lambda x: parabola_eval(qL, dq, q6, x), 1.0 - y, 1.0) / y
        left = quad(lambda x: parabola_eval(qL, dq, q6, x), 0.0, y) / y
        assert oracle.avg_right_part(qR, dq, q6, y) == pytest.approx(right, rel=1e-12, abs=1e-12)
        assert oracle.avg_left_part(qL, dq, q6, y) == pytest.approx(left, rel=1e-12, abs=1e-12)


# --------------------------------------------------------------- face Riemann (S2)

def test_riemann_equal_states():
    V, P = oracle.face_riemann(1.3, 1.3, 0.7, 0.7, 0.25, 0.25, 0.7, 0.7, 1.4)
    assert V == 0.25 and P == 0.7


def test_riemann_mirror_symmetry():
    """Swapping left and right and negating velocities negates V and keeps P."""
    rng = np.random.default_rng(14)
    for _ in range(100):
        rl, rr, pl, pr = rng.uniform(0.1, 5, 4)
        vl, vr = rng.normal(size=2)
        pls, prs = rng.uniform(0.1, 5, 2)
        V1, P1 = oracle.face_riemann(rl, rr, pl, pr, vl, vr, pls, prs, 1.4)
        V2, P2 = oracle.face_riemann(rr, rl, pr, pl, -vr, -vl, prs, pls, 1.4)
        assert V2 == pytest.approx(-V1, rel=1e-13, abs=1e-13)
        assert P2 == pytest.approx(P1, rel=1e-13)


@pytest.mark.parametrize("gamma", [1.4, 5.0 / 3.0])
def test_riemann_weak_waves_match_exact_star_state(gamma):
    """With piecewise-constant data the face solution is the acoustic (linearised)
    Riemann solution; for weak jumps of size eps it must agree with the exact star state
    to O(eps^2).  A missing impedance factor or a flipped sign is O(eps) and fails."""
    rng = np.random.default_rng(15)
    for _ in range(20):
        r0, p0 = rng.uniform(0.5, 2.0, 2)
        v0 = rng.normal()
        dr, dp, dv = rng.normal(size=3)
        errs = []
        for eps in (1e-2, 5e-3):
            rl, rr = r0 * (1 + eps * dr), r0 * (1 - eps * dr)
            pl, pr = p0 * (1 + eps * dp), p0 * (1 - eps * dp)
            vl, vr = v0 + eps * dv, v0 - eps * dv
            V, P = oracle.face_riemann(rl, rr, pl, pr, vl, vr, pl, pr, gamma)
            ps, us = exact.riemann_star(rl, vl, pl, rr, vr, pr, gamma)
            errs.append(max(abs(P - ps) / p0, abs(V - us) / math.sqrt(gamma * p0 / r0)))
        jump = 2e-2 * max(abs(dr), abs(dp), abs(dv), 0.1)
        assert errs[0] < 0.5 * jump ** 2 + 1e-12  # an O(eps) mistake is ~jump
        assert errs[1] < errs[0] * 0.35  # second order: halving eps quarters the error


def test_face_lambda_between_cell_sound_speeds():
    """The modified Roe average keeps lambda between the adjacent sound speeds, and at a
    dense/rarefied interface stays near the dense side's speed (Sec. 1.1 remark)."""
    rng = np.random.default_rng(16)
    g = 1.4
    for _ in range(200):
        rl, rr, pl, pr = np.exp(rng.uniform(-8, 3, 4))
        lam = oracle.face_lambda(rl, rr, pl, pr, g)
        cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
        assert min(cl, cr) * (1 - 1e-12) <= lam <= max(cl, cr) * (1 + 1e-12)
    # isothermal dense gas next to a 1e-8 rarer gas: lambda ~ the common sound speed
    lam = oracle.face_lambda(1.0, 1e-8, 1.0, 1e-8, 1.0)
    assert lam == pytest.approx(1.0, rel=1e-10)


# ------------------------------------------------------------- energy correction

def test_energy_correction_branches():
    """Sec. 'The conservation of total energy': the four cases of the correction."""
    # dense: rho eps = rho E - |m|^2 / (2 rho)
    u, code = oracle.energy_correction([2.0, 1.0, -2.0, 0.5, 5.0, 9.0], 1e-5)
    assert code == 0 and u[5] == pytest.approx(5.0 - (1 + 4 + 0.25) / 4.0)
    assert np.all(u[:5] == [2.0, 1.0, -2.0, 0.5, 5.0])
    # dense with non-positive difference: advected rho eps kept
    u, code = oracle.energy_correction([1.0, 3.0, 0.0, 0.0, 1.0, 0.25], 1e-5)
    assert code == 2 and u[5] == 0.25
    # vacuum: keep eps and direction, |v| = sqrt(2 (E - eps)) per unit mass
    rho = 1e-9
    u, code = oracle.energy_correction([rho, 3e-9, 4e-9, 0.0, 5e-9, 1e-9], 1e-5)
    v = np.array(u[1:4]) / rho
    assert code == 1 and u[5] == 1e-9
    assert np.linalg.norm(v) == pytest.approx(math.sqrt(2 * (5e-9 - 1e-9) / rho), rel=1e-13)
    assert v[0] / v[1] == pytest.approx(0.75, rel=1e-13)
    # vacuum with rho E < rho eps: momentum dropped, rho eps = rho E
    u, code = oracle.energy_correction([rho, 3e-9, 4e-9, 0.0, 1e-9, 2e-9], 1e-5)
    assert code == 3 and np.all(u[1:4] == 0.0) and u[5] == 1e-9


# ----------------------------------------------------------------- whole step

def test_cfl_closed_form():
    pb = inputs.uniform_flow(n=(8, 6, 5), v=(0.3, -0.4, 1.2), rho=2.0, p=3.0)
    g = grid_of(pb)
    dt = oracle.cfl_dt(g, pb.u)
    c = math.sqrt(1.4 * 3.0 / 2.0)
    vmag = math.sqrt(0.09 + 0.16 + 1.44)
    assert dt == pytest.approx(0.2 * min(pb.h) / (vmag + c), rel=1e-14)


def test_uniform_flow_unchanged():
    """Galilean uniform flow: flat parabolas, equal fluxes, nothing changes."""
    pb = inputs.uniform_flow()
    g = grid_of(pb)
    u = pb.u
    for _ in range(3):
        u, dg = oracle.step(g, u, oracle.cfl_dt(g, u))
    for a, b in zip(u, pb.u):
        assert np.max(np.abs(a - b)) <= 1e-14 * max(1.0, np.max(np.abs(b)))


def test_conservation_periodic_random():
    """Periodic box: mass, momentum and total energy are conserved to round-off (both
    stages are in flux form; a lost or doubled face term breaks this)."""
    pb = inputs.random_smooth(n=(12, 10, 8))
    g = grid_of(pb)
    s0 = oracle.diagnostics(g, pb.u)["sums"]
    u = pb.u
    for _ in range(4):
        u, dg = oracle.step(g, u, oracle.cfl_dt(g, u))
    assert dg["n_vacuum"] == 0
    for f in range(5):
        scale = max(abs(s0[0]), abs(s0[4]))
        assert abs(dg["sums"][f] - s0[f]) <= 2e-14 * scale


def test_conservation_rough_data():
    pb = inputs.random_rough(n=(10, 9, 8), bc=(1,) * 6)
    g = grid_of(pb)
    s0 = oracle.diagnostics(g, pb.u)["sums"]
    u, dg = oracle.step(g, pb.u, 0.5 * oracle.cfl_dt(g, pb.u))
    for f in range(5):
        assert abs(dg["sums"][f] - s0[f]) <= 1e-13 * max(abs(s0[0]), abs(s0[4]))


def test_planar_data_stays_planar_and_matches_1d():
    """Data uniform in y and z stays bitwise uniform and equals the 1D run."""
    n = 32
    p3 = inputs.planar_sod_3d(n)
    p3.u = [a[:6, :5, :].copy() for a in p3.u]
    p3.n = (n, 5, 6)
    g3 = grid_of(p3)
    p1 = inputs.sod_1d(n, cfl=0.2)
    g1 = grid_of(p1)
    u3, u1 = p3.u, p1.u
    for _ in range(10):
        tau = oracle.cfl_dt(g1, u1)
        u3, _ = oracle.step(g3, u3, tau)
        u1, _ = oracle.step(g1, u1, tau)
    for f in range(6):
        assert np.all(u3[f] == u3[f][:1, :1, :])
    for f in (0, 1, 4, 5):
        d = np.abs(u3[f][0, 0] - u1[f][0, 0]).sum() / max(np.abs(u1[f]).sum(), 1e-300)
        assert d <= 1e-12


def test_point_blast_mirror_and_permutation_symmetry():
    """A blast centred in the box is symmetric under x -> -x and under axis exchange."""
    pb = inputs.point_blast_3d(n=16)
    g = grid_of(pb)
    u = pb.u
    for _ in range(6):
        u, dg = oracle.step(g, u, oracle.cfl_dt(g, u))
    rho, mx, my, mz, en, ei = u
    scale = np.max(np.abs(en))
    assert np.max(np.abs(rho - rho[:, :, ::-1])) <= 1e-12 * np.max(rho)
    assert np.max(np.abs(mx + mx[:, :, ::-1])) <= 1e-12 * np.max(np.abs(mx))
    assert np.max(np.abs(en - en[::-1, :, :])) <= 1e-12 * scale
    assert np.max(np.abs(rho - np.transpose(rho, (0, 2, 1)))) <= 1e-12 * np.max(rho)
    assert np.max(np.abs(mx - np.transpose(my, (0, 2, 1)))) <= 1e-12 * np.max(np.abs(mx))
    assert np.max(np.abs(rho - np.transpose(rho, (2, 1, 0)))) <= 1e-12 * np.max(rho)


def _sod_l1(n, row=1):
    pb = inputs.sod_1d(n, row=row)
    g = grid_of(pb)
    u, t, steps, dg = oracle.run(g, pb.u, pb.t_end)
    edges = np.arange(n + 1) / n
    ex = exact.riemann_cell_averages(*pb.extra["states"], pb.gamma, pb.extra["x_split"], t,
                                     edges, sub=8)
    return np.mean(np.abs(u[0].ravel() - ex[0])), u, dg


def test_sod_converges_to_exact_solution():
    """Table 2 row 1 against the exact Riemann solution: L1(rho) falls under refinement,
    and at 256 cells stays below the bound registered from the first oracle run
    (2.55e-3 measured; bound 3.5e-3)."""
    e100, _, _ = _sod_l1(100)
    e200, _, _ = _sod_l1(200)
    e256, u, dg = _sod_l1(256)
    assert e200 < 0.7 * e100
    assert e256 < 3.5e-3
    assert dg["n_nonphys"] == 0
    # conserved to round-off: the boundary states stay static, the momentum gain is
    # exactly (p_L - p_R) t
    assert dg["sums"][0] == pytest.approx(0.5625, rel=1e-14)
    assert dg["sums"][4] == pytest.approx(1.375, rel=1e-14)
    assert dg["sums"][1] == pytest.approx(0.9 * 0.2, rel=1e-12)


@pytest.mark.parametrize("row", [2, 3])
def test_table2_rows_2_3_positive_and_close(row):
    """Rows 2 (strong rarefactions) and 3 (pressure ratio 1e5) stay physical and close to
    the exact solution in L1."""
    e, u, dg = _sod_l1(256, row=row)
    assert dg["n_nonphys"] == 0
    scale = {2: 0.05, 3: 0.12}[row]
    assert e < scale


def test_sod_shock_width_two_to_three_cells():
    """Sec. 'The Sod shock-tube problem': the high-order shock spans about two cells
    (100 cells, t = 0.2).  Measured as the 10-90% rise of rho across the shock."""
    n = GOLDEN["shock_tubes"]["cells"]
    pb = inputs.sod_1d(n)
    g = grid_of(pb)
    u, t, steps, dg = oracle.run(g, pb.u, pb.t_end)
    rho = u[0].ravel()
    ps, us = exact.riemann_star(*pb.extra["states"], pb.gamma)
    # post-shock density from the exact solution
    r_post = exact.riemann_sample(*pb.extra["states"], pb.gamma, np.array([us + 1e-9]))[0][0]
    lo, hi = 0.125, r_post
    x = (np.arange(n) + 0.5) / n
    window = (x > 0.75) & (x < 0.95)
    r = rho[window]
    f = (r - lo) / (hi - lo)
    width = np.sum((f > 0.1) & (f < 0.9))
    assert width <= GOLDEN["shock_width_cells"]["high_order"] + 1


def _advected_error(n):
    pb = inputs.advected_wave(n)
    g = grid_of(pb)
    u, t, steps, dg = oracle.run(g, pb.u, 1.0)
    ex = exact.advected_wave_exact(pb.extra["edges"], t)
    return np.mean(np.abs(u[0].ravel() - ex))


def test_advected_wave_order():
    """Smooth density wave advected one period (exact = translation): L1 order >= 1.5."""
    e32, e64 = _advected_error(32), _advected_error(64)
    order = math.log2(e32 / e64)
    assert order >= 1.5, order


def test_aksenov_order():
    """Sec. 'The Aksenov Test': T = log2(E_{N/2}/E_N) on density at N = 628, t = pi/2,
    at the paper's CFL = 0.2.  The paper prints T = 1.713.  The scheme as the paper states
    it advances the Eulerian and Lagrangian stages one after the other with forward
    differences in time (its conclusion calls the time discretisation simple), so with
    tau proportional to h its error is O(tau) = O(h): the oracle measures T = 1.08 and the
    error halves when CFL halves at fixed N (checked below).  The pin is therefore first
    order, 0.9 <= T <= 1.3, plus the O(tau) signature; the paper's 1.713 is recorded as
    not reproduced.  A dropped or mis-signed term stops convergence (T ~ 0) or blows up."""
    errs = {}
    for n, cfl in ((314, 0.2), (628, 0.2), (314, 0.1)):
        pb = inputs.aksenov(n, cfl=cfl)
        g = grid_of(pb)
        u, t, steps, dg = oracle.run(g, pb.u, pb.t_end)
        rho_ex, _ = exact.aksenov_cell_averages(pb.extra["edges"], t)
        errs[(n, cfl)] = np.sum(np.abs(u[0].ravel() - rho_ex)) * pb.h[0]
    T = math.log2(errs[(314, 0.2)] / errs[(628, 0.2)])
    assert 0.9 <= T <= 1.3, (T, errs)
    assert errs[(314, 0.1)] < 0.75 * errs[(314, 0.2)]
    assert errs[(628, 0.2)] < 3e-3


def test_acoustic_wave_first_order_in_time_high_order_in_space():
    """Small-amplitude sound wave, one period.  Pure advection (test_advected_wave_order)
    converges at order > 2; acoustics couples both stages and converges at first order
    with an error proportional to CFL, the splitting's signature."""
    def err(n, cfl, eps=1e-6, g=1.4):
        h = 1.0 / n
        edges = np.arange(n + 1) * h
        k = 2 * math.pi
        avg = (np.cos(k * edges[:-1]) - np.cos(k * edges[1:])) / (k * h)
        c = math.sqrt(g)
        u = inputs.conserved((1 + eps * avg)[None, None, :], (c * eps * avg)[None, None, :], 0.0,
                             0.0, (1 + g * eps * avg)[None, None, :], g)
        G = oracle.Grid((n, 1, 1), (h, 1.0, 1.0), g, (1, 1, 0, 0, 0, 0), cfl, rho_mean=1.0)
        out, t, steps, dg = oracle.run(G, u, 1.0 / c)
        return np.mean(np.abs(out[0].ravel() - (1 + eps * avg))) / eps
    e32, e64, e32h = err(32, 0.4), err(64, 0.4), err(32, 0.2)
    assert 0.85 <= math.log2(e32 / e64) <= 1.3
    assert 0.4 <= e32h / e32 <= 0.65


def test_vacuum_expansion_conserves_total_energy():
    """Sec. 'The expansion of gas into vacuum': total energy constant to round-off while
    kinetic energy rises and internal energy falls.  The printed scheme survives a density
    contrast of 1e-2 but not 1e-3 (the acoustic face solve, with one impedance from the
    dense side, pushes a nearly empty cell with about half the dense pressure), so the
    ambient gas is at 1e-2 and the vacuum threshold is raised to 0.3 x mean density so
    that the vacuum branch of the energy correction runs."""
    pb = inputs.vacuum_sphere(n=20, rho_vac=1e-2, p_vac=1e-2)
    pb.bc = (1,) * 6  # periodic: nothing leaves the box
    g = grid_of(pb)
    g.vacuum_frac = 0.3
    u = pb.u
    d0 = oracle.diagnostics(g, u)
    kin = []
    nvac = 0
    for _ in range(12):
        u, dg = oracle.step(g, u, oracle.cfl_dt(g, u))
        nvac += dg["n_vacuum"]
        kin.append(np.sum((u[1] ** 2 + u[2] ** 2 + u[3] ** 2) / (2 * u[0])))
    assert nvac > 0 and dg["n_nonphys"] == 0
    # 12 steps of 8000 cells: round-off of the sums, ~1e-14 relative per step
    assert abs(dg["sums"][4] - d0["sums"][4]) <= 1e-12 * d0["sums"][4]
    assert dg["sums"][0] == pytest.approx(d0["sums"][0], rel=1e-12)
    assert kin[-1] > kin[0] > 0
    assert dg["sums"][5] < d0["sums"][5]


@pytest.mark.slow
def test_point_blast_radius_matches_sedov():
    """Point blast (Sec. 'The Sedov blast wave' setup with gamma = 5/3): the radius of the
    density peak follows R = xi0 (E t^2/rho0)^(1/5) within two cells, xi0 from the
    self-similar solution."""
    n = 32
    xi0 = exact.sedov_xi0(5.0 / 3.0)
    pb = inputs.point_blast_3d(n=n, radius_end=0.3, xi0=xi0)
    g = grid_of(pb)
    u, t, steps, dg = oracle.run(g, pb.u, pb.t_end)
    h = pb.h[0]
    c = (np.arange(n) + 0.5) * h - 0.5
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(x * x + y * y + z * z).ravel()
    rho = u[0].ravel()
    bins = np.arange(0, 0.5, h)
    idx = np.digitize(r, bins)
    prof = np.array([rho[idx == i].mean() if np.any(idx == i) else 0 for i in range(1, len(bins))])
    r_peak = bins[np.argmax(prof)] + 0.5 * h
    R = xi0 * (1.0 * t * t / 1.0) ** 0.2
    assert abs(r_peak - R) <= 2.0 * h, (r_peak, R)


# ------------------------------------------------------------------- Poisson (S12)

def test_poisson_solution_satisfies_the_printed_stencil():
    """The harmonic-space solve inverts eq. stencil27point: applying the printed 27-point
    weights (-38/9, 4/9, 1/9, 1/36) to Phi gives 4 pi G h^2 (rho - mean rho) to round-off.
    A wrong sign, a missing 2/3 or a transposed axis in the symbol fails this."""
    from oracle import poisson
    rng = np.random.default_rng(21)
    rho = rng.uniform(0.5, 2.0, size=(12, 10, 16))
    h, G = 0.05, 1.3
    phi = poisson.solve_periodic(rho, h, G)
    lhs = poisson.apply_stencil(phi)
    rhs = 4.0 * math.pi * G * h * h * (rho - rho.mean())
    assert np.max(np.abs(lhs - rhs)) <= 1e-12 * np.max(np.abs(rhs))
    assert abs(phi.mean()) <= 1e-14 * np.max(np.abs(phi))


def test_poisson_converges_to_the_continuous_potential():
    """For rho = sin(2 pi x) sin(2 pi y) sin(2 pi z) the continuum potential is
    -4 pi G rho / (3 (2 pi)^2); the discrete solution converges at second order or better."""
    from oracle import poisson
    errs = []
    for n in (16, 32):
        h = 1.0 / n
        c = (np.arange(n) + 0.5) * h
        z, y, x = np.meshgrid(c, c, c, indexing="ij")
        rho = np.sin(2 * math.pi * x) * np.sin(2 * math.pi * y) * np.sin(2 * math.pi * z)
        exact = -4 * math.pi * rho / (3 * (2 * math.pi) ** 2)
        errs.append(np.max(np.abs(poisson.solve_periodic(rho, h) - exact)))
    assert math.log2(errs[0] / errs[1]) >= 1.9


# ------------------------------------------------------------ scheme variants (NEXT)

def _sod_widths(flags, n=100):
    pb = inputs.sod_1d(n, cfl=0.2)
    g = oracle.Grid(pb.n, pb.h, pb.gamma, pb.bc, pb.cfl, rho_mean=1.0, flags=flags)
    u, t, steps, dg = oracle.run(g, pb.u, pb.t_end)
    rho = u[0].ravel()
    x = (np.arange(n) + 0.5) / n
    states = pb.extra["states"]
    ps, us = exact.riemann_star(*states, pb.gamma)
    r_post = exact.riemann_sample(*states, pb.gamma, np.array([us + 1e-9]))[0][0]
    r_cl = exact.riemann_sample(*states, pb.gamma, np.array([us - 1e-9]))[0][0]

    def width(lo, hi, sel):
        f = (rho[sel] - lo) / (hi - lo)
        return int(np.sum((f > 0.1) & (f < 0.9)))
    return width(0.125, r_post, (x > 0.7) & (x < 0.99)), width(r_post, r_cl, (x > 0.5) & (x < 0.8))


def test_first_order_variant_is_more_diffusive():
    """Sec. 'The Sod shock-tube problem': the paper reports the shock spread over 12 cells
    with the first-order scheme and 2 with the high-order one (100 cells).  The oracle's
    first-order variant (piecewise-constant face problems, Sec. 1.1) spreads the shock over 4
    and the contact over 12 cells (10-90 %), against 2 and 3 with PPML."""
    shock_hi, contact_hi = _sod_widths(0)
    shock_fo, contact_fo = _sod_widths(oracle.FIRST_ORDER)
    assert shock_hi <= GOLDEN["shock_width_cells"]["high_order"] + 1
    assert shock_fo >= 2 * shock_hi
    assert contact_fo >= 8 and contact_fo >= 3 * contact_hi


def test_nine_point_template_reduces_grid_alignment_artifacts():
    """Sec. 1.3 (rotating disk p = rho = 2 - r, omega = 1 inside r = 1): the 9-point
    velocity template removes the artifacts of the 1-point face velocity.  Measured as the
    non-axisymmetric residual of rho about its ring means at t = 0.5 on a 48^2 grid."""
    n, L = 48, 3.0
    h = L / n
    c = (np.arange(n) + 0.5) * h - L / 2
    y, x = np.meshgrid(c, c, indexing="ij")
    r = np.sqrt(x * x + y * y)
    inside = r < 1.0
    rho = np.where(inside, 2.0 - r, 1.0)
    om = np.where(inside, 1.0, 0.0)
    u0 = inputs.conserved(rho[None], (-om * y)[None], (om * x)[None], 0.0, rho[None], 1.4)
    res = {}
    for flags in (0, oracle.VHAT_1PT):
        g = oracle.Grid((n, n, 1), (h, h, 1.0), 1.4, (0,) * 6, 0.2, rho_mean=1.0, flags=flags)
        u, t, steps, dg = oracle.run(g, u0, 0.5)
        rr = u[0][0]
        rb = np.floor(r / 0.05).astype(int)
        resid = rr.copy()
        for k in np.unique(rb):
            resid[rb == k] -= rr[rb == k].mean()
        res[flags] = np.abs(resid[r < 1.1]).mean()
    assert res[oracle.VHAT_1PT] > 1.15 * res[0], res


def _delta_state(n, axis, centre, delta=1.0):
    """Uniform gas at rest (rho = 1, p = 1) with momentum `delta` along `axis` in one cell."""
    shape = (n[2], n[1], n[0])
    rho = np.ones(shape)
    m = [np.zeros(shape) for _ in range(3)]
    m[axis][centre[2], centre[1], centre[0]] = delta
    return [rho, m[0], m[1], m[2], np.full(shape, 2.5), np.full(shape, 2.5)]


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_velocity_template_weights_on_a_delta(axis):
    """Eq. veltemplate: the transverse template puts 1/16 on the four corner neighbours,
    1/8 on the four edge neighbours and 1/4 on the cell itself (the weights the paper
    prints, tests/golden/paper_values.json); with uniform density the face velocity of eq.
    modspaceaveragevelocitylagrange is the mean of the two adjacent template values.  A
    delta of v_a in one cell therefore gives v hat = w/2 on the two faces of that cell's
    line and of its transverse neighbours' lines (w the template weight of the line) and
    zero on every other face.  Swapping the corner and edge weights (which still sum to
    one) or the template's transverse axes fails this."""
    w = GOLDEN["velocity_template"]
    n, c = (7, 8, 9), (3, 4, 4)
    g = oracle.Grid(n, (1.0, 1.0, 1.0), 1.4, (1,) * 6, 0.2)
    vh = oracle.face_velocities(g, _delta_state(n, axis, c), axis)
    expect = np.zeros_like(vh)
    tr = [a for a in range(3) if a != axis]
    for db in (-1, 0, 1):
        for dc in (-1, 0, 1):
            k = abs(db) + abs(dc)
            wt = w["centre"] if k == 0 else (w["edge"] if k == 1 else w["corner"])
            for face in (c[axis], c[axis] + 1):  # the two faces of the delta's cell
                idx = list(c)
                idx[axis] = face
                idx[tr[0]] += db
                idx[tr[1]] += dc
                expect[idx[2], idx[1], idx[0]] = 0.5 * wt
    assert np.allclose(vh, expect, rtol=0, atol=1e-15)
    assert vh.sum() == pytest.approx(1.0, abs=1e-14)  # the weights sum to one per face plane


def test_velocity_template_one_point_and_lower_dimensional_marginals():
    """The one-point variant (Sec. 1.3) takes the cell's own v; on a 2D grid the template
    of the remaining transverse axis is the marginal of the 9-point one (1/4, 1/2, 1/4:
    the corner and edge weights summed over the inactive axis) and in 1D it is v itself."""
    n, c = (9, 9, 1), (4, 4, 0)
    g = oracle.Grid(n, (1.0, 1.0, 1.0), 1.4, (1, 1, 1, 1, 0, 0), 0.2)
    vh = oracle.face_velocities(g, _delta_state(n, 0, c), 0)[0]
    w = GOLDEN["velocity_template"]
    side, mid = 2 * w["corner"] + w["edge"], 2 * w["edge"] + w["centre"]
    assert (side, mid) == (0.25, 0.5)
    expect = np.zeros_like(vh)
    for face in (4, 5):
        expect[3, face] = expect[5, face] = 0.5 * side
        expect[4, face] = 0.5 * mid
    assert np.allclose(vh, expect, rtol=0, atol=1e-15)
    g1 = oracle.Grid(n, (1.0, 1.0, 1.0), 1.4, (1, 1, 1, 1, 0, 0), 0.2, flags=oracle.VHAT_1PT)
    vh1 = oracle.face_velocities(g1, _delta_state(n, 0, c), 0)[0]
    expect1 = np.zeros_like(vh1)
    expect1[4, 4] = expect1[4, 5] = 0.5
    assert np.allclose(vh1, expect1, rtol=0, atol=1e-15)
    n1 = (9, 1, 1)
    g2 = oracle.Grid(n1, (1.0, 1.0, 1.0), 1.4, (1, 1, 0, 0, 0, 0), 0.2)
    vh2 = oracle.face_velocities(g2, _delta_state(n1, 0, (4, 0, 0)), 0)[0, 0]
    assert np.allclose(vh2, [0, 0, 0, 0, 0.5, 0.5, 0, 0, 0, 0], rtol=0, atol=1e-15)


def test_face_velocity_roe_weights():
    """Eq. modspaceaveragevelocitylagrange: v hat = (v_i sqrt(rho_i) + v_i+1 sqrt(rho_i+1)) /
    (sqrt(rho_i) + sqrt(rho_i+1)).  A 1D line with rho = 1 | 4 and v = 0.3 | 0.9 gives
    (0.3 + 2 * 0.9) / 3 = 0.7 at the interface (swapped weights: 0.5) and the adjacent
    cells' own v elsewhere."""
    n = (12, 1, 1)
    rho = np.where(np.arange(12) < 6, 1.0, 4.0)
    v = np.where(np.arange(12) < 6, 0.3, 0.9)
    z = np.zeros(12)
    u = [rho[None, None], (rho * v)[None, None], z[None, None], z[None, None],
         np.full((1, 1, 12), 3.0), np.full((1, 1, 12), 1.0)]
    g = oracle.Grid(n, (1.0, 1.0, 1.0), 1.4, (0,) * 6, 0.2)
    vh = oracle.face_velocities(g, u, 0)[0, 0]
    assert vh[6] == pytest.approx(0.7, abs=1e-15)
    assert np.allclose(vh[:6], 0.3, rtol=0, atol=1e-15)
    assert np.allclose(vh[7:], 0.9, rtol=0, atol=1e-15)


def _gravity_case(m0, gvec, tau=0.01, n=12, rho=1.3, p=1.0, gamma=1.4):
    """Uniform gas (momentum m0) in the linear potential Phi = g . x on an n^3 outflow grid:
    one oracle step.  Returns (input, output) restricted to cells at least 4 from every
    face, which no boundary value reaches in either stage."""
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    zz, yy, xx = np.meshgrid(x, x, x, indexing="ij")
    phi = gvec[0] * xx + gvec[1] * yy + gvec[2] * zz
    shape = (n, n, n)
    e = p / (gamma - 1.0)
    ke = 0.5 * sum(mc * mc for mc in m0) / rho
    u = [np.full(shape, rho)] + [np.full(shape, mc) for mc in m0] + \
        [np.full(shape, e + ke), np.full(shape, e)]
    g = oracle.Grid((n, n, n), (h, h, h), gamma, (0,) * 6, 0.2, rho_mean=rho)
    out, _ = oracle.step(g, u, tau, phi=phi)
    core = (slice(4, n - 4),) * 3
    return [f[core] for f in u], [f[core] for f in out]


def test_gravity_source_of_gas_at_rest():
    """Model equations, source terms -rho grad Phi (momentum) and -rho v . grad Phi (total
    energy), central difference of Phi (reading G16): uniform gas at rest in Phi = g . x
    gains momentum -tau rho g in one step, exactly up to rounding, and keeps its total
    energy (the flow it gains is uniform, so the Lagrangian fluxes cancel).  A flipped sign
    or a missing 1/2 in the central difference fails."""
    gvec, tau, rho = (0.3, -0.2, 0.5), 0.01, 1.3
    uin, uout = _gravity_case((0.0, 0.0, 0.0), gvec, tau=tau, rho=rho)
    assert np.allclose(uout[0], rho, rtol=1e-15, atol=0)
    for a in range(3):
        assert np.allclose(uout[1 + a], -tau * rho * gvec[a], rtol=1e-10, atol=0), a
    assert np.allclose(uout[4], uin[4], rtol=1e-15, atol=0)
    # the energy correction takes the new kinetic energy from the internal energy
    ke = 0.5 * tau * tau * rho * sum(gc * gc for gc in gvec)
    assert np.allclose(uout[5], uin[5] - ke, rtol=1e-12, atol=0)


def test_gravity_source_of_moving_gas():
    """With uniform momentum m the total energy changes by -tau m . g in one step (the
    work of gravity on the flow, taken from U^n), the momentum by -tau rho g."""
    m0, gvec, tau, rho = (0.4, 0.1, -0.3), (0.3, -0.2, 0.5), 0.01, 1.3
    uin, uout = _gravity_case(m0, gvec, tau=tau, rho=rho)
    work = -tau * sum(mc * gc for mc, gc in zip(m0, gvec))
    assert np.allclose(uout[4] - uin[4], work, rtol=1e-9, atol=0)
    for a in range(3):
        assert np.allclose(uout[1 + a], m0[a] - tau * rho * gvec[a], rtol=1e-12, atol=0), a


# ------------------------------------------------------- reflecting walls (NEXT)

def _local_peaks(q, x, order=40):
    return [(x[i], q[i]) for i in range(order, len(q) - order)
            if q[i] == q[i - order:i + order + 1].max()]


@pytest.mark.slow
def test_two_interacting_blast_waves():
    """The paper's two-blast-wave test (2400 cells, reflecting walls): the density peak about
    6.5 near x = 0.76, the precursor about 1.0 near x = 0.86 and velocity peaks near x = 0.65
    and 0.86, as printed; reflecting walls conserve mass and total energy to round-off."""
    gv = GOLDEN["two_blast_waves"]
    pb = inputs.two_blast_waves(gv["cells"])
    g = grid_of(pb)
    u, t, steps, dg = oracle.run(g, pb.u, pb.t_end)
    assert t == pb.t_end and dg["n_nonphys"] == 0
    x = (np.arange(pb.n[0]) + 0.5) * pb.h[0]
    rho = u[0].ravel()
    v = u[1].ravel() / rho
    i = int(np.argmax(rho))
    assert abs(rho[i] - gv["shock"]["rho"]) <= 0.3 and abs(x[i] - gv["shock"]["x"]) <= 0.02
    pre = [(xx, q) for xx, q in _local_peaks(rho, x) if abs(xx - gv["precursor"]["x"]) <= 0.015]
    assert pre and abs(pre[0][1] - gv["precursor"]["rho"]) <= 0.1, pre
    vp = [xx for xx, q in _local_peaks(v, x) if q > 1.0]
    assert len(vp) == 2 and all(abs(a - b) <= 0.015 for a, b in zip(vp, gv["velocity_peaks_x"])), vp
    s0 = oracle.diagnostics(g, pb.u)["sums"]
    assert dg["sums"][0] == pytest.approx(s0[0], rel=1e-13)
    assert dg["sums"][4] == pytest.approx(s0[4], rel=1e-13)


# ------------------------------------------------ isolated Poisson solve (NEXT, S12)

def _table1_case(n, printed_rhs=False):
    """Table 1 profile on [-1, 1]^3 (sphere inscribed), relative max error of Phi."""
    from oracle import poisson
    h = 2.0 / n
    c = poisson.cell_centres(n, h)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(x * x + y * y + z * z)
    rho = np.where(r <= 1.0, 2 * r ** 3 - 3 * r ** 2 + 1, 0.0)
    exact_phi = np.where(r <= 1.0, 4 * math.pi / 15 * r ** 5 - 3 * math.pi / 5 * r ** 4
                         + 2 * math.pi / 3 * r ** 2 - 3 * math.pi / 5, -4 * math.pi / (15 * r))
    phi = poisson.solve_isolated(rho, h, 1.0, printed_rhs=printed_rhs)
    return np.max(np.abs(phi - exact_phi)) / np.max(np.abs(exact_phi))


def test_table1_potential_needs_the_corrected_density():
    """The printed potential solves Delta Phi = 4 pi rho for rho = 2r^3 - 3r^2 + 1, not for
    the printed 2r^3 - 2r^2 + 1 (the radial Laplacian of each polynomial piece, with Phi and
    Phi' continuous at r = 1 and the exterior mass 4 pi / 15 equal to the integral of rho)."""
    P = np.polynomial.Polynomial
    inner = P([-3 * math.pi / 5, 0, 2 * math.pi / 3, 0, -3 * math.pi / 5, 4 * math.pi / 15])
    r = np.linspace(0.05, 1.0, 40)
    lap = inner.deriv(2)(r) + 2.0 * inner.deriv(1)(r) / r
    assert np.allclose(lap / (4 * math.pi), 2 * r ** 3 - 3 * r ** 2 + 1, rtol=0, atol=1e-12)
    assert not np.allclose(lap / (4 * math.pi), 2 * r ** 3 - 2 * r ** 2 + 1, atol=1e-3)
    assert abs(inner(1.0) + 4 * math.pi / 15) < 1e-14           # Phi continuous
    assert abs(inner.deriv(1)(1.0) - 4 * math.pi / 15) < 1e-14  # Phi' = M / r^2 continuous
    mass = 4 * math.pi * (P([1, 0, -3, 2]) * P([0, 0, 1])).integ()(1.0)
    assert abs(mass - 4 * math.pi / 15) < 1e-14


def test_multipole_boundary_two_masses_closed_form():
    """Two unit masses at (+-d, 0, 0): the exact far field is -sum m / |r - r_j|.  The
    monopole + quadrupole boundary value (MacCullagh, with the 1/2) differs from it by
    O(R^-5); the monopole alone, or the quadrupole without the 1/2, by O(R^-3)."""
    from oracle import poisson
    n, h = 7, 1.0
    rho = np.zeros((n, n, n))
    rho[3, 3, 1] = rho[3, 3, 5] = 1.0  # cells centred at x = -2 and +2
    mom = poisson.multipole_moments(rho, h)
    assert mom[0] == 2.0 and mom[1] == 0.0 and mom[2] == 8.0 and mom[3] == 8.0
    dirs = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1 / math.sqrt(2), 1 / math.sqrt(2), 0)]
    errs = {}
    for R in (40.0, 80.0):
        for dv in dirs:
            x, y, z = (R * c for c in dv)
            exact_phi = -1.0 / math.dist((x, y, z), (-2, 0, 0)) - 1.0 / math.dist((x, y, z), (2, 0, 0))
            mp = float(poisson.multipole_potential(mom, x, y, z))
            mono = -2.0 / R
            no_half = mono + 2.0 * (mp - mono)
            errs[(R, dv)] = abs(mp - exact_phi)
            assert abs(mp - exact_phi) <= 0.01 * abs(mono - exact_phi)
            assert abs(mp - exact_phi) <= 0.01 * abs(no_half - exact_phi)
        # on the axis, MacCullagh gives -2m/R - 2 m d^2 / R^3
    assert abs(float(poisson.multipole_potential(mom, 40.0, 0, 0)) - (-2 / 40 - 8 / 40 ** 3)) < 1e-15
    for dv in dirs:
        assert errs[(40.0, dv)] / errs[(80.0, dv)] >= 24.0  # R^-5


def test_multipole_boundary_random_symmetric_blob():
    """A point-symmetric random mass distribution (no dipole, no octupole): the boundary
    value approaches the direct sum as R^-5 in every direction, which needs the products of
    inertia with the right sign in I_0."""
    from oracle import poisson
    rng = np.random.default_rng(5)
    rho = rng.uniform(0.0, 1.0, size=(5, 7, 9))
    rho = rho + rho[::-1, ::-1, ::-1]
    rho[:, :4, :5] *= 3.0  # anisotropic, with products of inertia
    rho = rho + rho[::-1, ::-1, ::-1]
    h = 0.5
    mom = poisson.multipole_moments(rho, h)
    assert abs(mom[4]) > 0.1 * mom[1]  # I_xy matters
    z, y, x = np.meshgrid(poisson.cell_centres(5, h), poisson.cell_centres(7, h),
                          poisson.cell_centres(9, h), indexing="ij")
    m = rho * h ** 3
    for dv in rng.normal(size=(6, 3)):
        dv = dv / np.linalg.norm(dv)
        e = []
        for R in (30.0, 60.0):
            p = R * dv
            direct = -np.sum(m / np.sqrt((p[0] - x) ** 2 + (p[1] - y) ** 2 + (p[2] - z) ** 2))
            e.append(abs(float(poisson.multipole_potential(mom, *p)) - direct))
        assert e[0] / e[1] >= 20.0, e


def test_isolated_solve_against_dense_solve_and_the_stencil():
    """Brute force on a 5x3x4 grid: the 60x60 matrix of the printed 27-point stencil with the
    shell moved to the right-hand side, solved densely, equals the sine-transform solve; and
    Phi extended by the multipole shell satisfies the stencil with 4 pi G h^2 (rho + D7 rho/12)
    (rho = 0 outside) to round-off."""
    from oracle import poisson
    rng = np.random.default_rng(8)
    shape = (4, 3, 5)
    rho = rng.uniform(0.1, 2.0, size=shape)
    h, G = 0.3, 1.7
    w = {1: 4.0 / 9.0, 2: 1.0 / 9.0, 3: 1.0 / 36.0}
    cells = [(k, j, i) for k in range(4) for j in range(3) for i in range(5)]
    A = np.zeros((60, 60))
    for row, (k, j, i) in enumerate(cells):
        A[row, row] = -38.0 / 9.0
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    nnz = abs(dx) + abs(dy) + abs(dz)
                    kk, jj, ii = k + dz, j + dy, i + dx
                    if nnz and 0 <= kk < 4 and 0 <= jj < 3 and 0 <= ii < 5:
                        A[row, cells.index((kk, jj, ii))] = w[nnz]
    rhs, shell = poisson.isolated_rhs(rho, h, G)
    dense = np.linalg.solve(A, rhs.reshape(-1)).reshape(shape)
    phi = poisson.solve_isolated(rho, h, G)
    assert np.max(np.abs(phi - dense)) <= 1e-12 * np.max(np.abs(dense))
    # residual with the shell: ghost values from the expansion at the ghost centres
    full = shell.copy()
    full[1:-1, 1:-1, 1:-1] = phi
    lhs = np.zeros(shape)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                nnz = abs(dx) + abs(dy) + abs(dz)
                wt = -38.0 / 9.0 if nnz == 0 else w[nnz]
                lhs += wt * full[1 + dz:5 + dz, 1 + dy:4 + dy, 1 + dx:6 + dx]
    rp = np.pad(rho, 1)
    d7 = sum(np.roll(rp, s, axis=a) for a in range(3) for s in (1, -1))[1:-1, 1:-1, 1:-1] - 6 * rho
    src = 4 * math.pi * G * h * h * (rho + d7 / 12.0)
    assert np.max(np.abs(lhs - src)) <= 1e-12 * np.max(np.abs(src))
    # the ghost centres are the cells just outside the grid: the corner ghost of the shell
    gx = poisson.cell_centres(7, h)[0]
    assert abs(gx - (-0.5 * 5 * h - 0.5 * h)) < 1e-15


def test_isolated_poisson_fourth_order_as_table1():
    """Table 1: the relative error of the analytic test drops about 16x per doubling (fourth
    order).  The oracle, on [-1, 1]^3 with the multipole boundary, drops it by 10-30x per
    doubling and is within a factor 3 of the paper's error at 16^3; with the right-hand side
    exactly as printed the drop is 4x (second order)."""
    tab = GOLDEN["poisson_table1"]
    e = [_table1_case(n) for n in (16, 32, 64)]
    for a, b in zip(e, e[1:]):
        assert 10.0 <= a / b <= 30.0, e
    paper16 = tab["relative_error"][0]
    assert paper16 / 3.0 <= e[0] <= 3.0 * paper16, (e[0], paper16)
    for pa, pb in zip(tab["relative_error"], tab["relative_error"][1:]):
        assert 15.0 <= pa / pb <= 17.0  # the golden values themselves are fourth order
    p = [_table1_case(n, printed_rhs=True) for n in (16, 32)]
    assert 3.5 <= p[0] / p[1] <= 4.5, p


# ------------------------------------------------------- disk Fourier amplitudes (NEXT)

def test_fourier_amplitudes_axisymmetric_disk_is_zero():
    """An axisymmetric disk has all A_m = 0 (the paper's statement).  On a square grid
    centred on the axis the sum over the four quarter-turn images of a column cancels
    e^{i m phi} exactly unless m is a multiple of 4, so those amplitudes vanish to
    round-off; A_4 and A_8 only carry the grid's own anisotropy."""
    from oracle import disk
    n, h = 96, 1.0 / 96
    c = (np.arange(n) + 0.5 - 0.5 * n) * h
    z, y, x = np.meshgrid(c[:8], c, c, indexing="ij")
    r = np.sqrt(x * x + y * y)
    rho = np.exp(-r / 0.125) * np.exp(-(z / 0.02) ** 2) + 1e-6
    a = disk.fourier_amplitudes(rho, h, 0.25, 8)
    for m in range(1, 9):
        if m % 4:
            assert a[m - 1] < 1e-13, (m, a[m - 1])
        else:
            assert a[m - 1] < 1e-2, (m, a[m - 1])


@pytest.mark.parametrize("m0", [2, 3, 7])
def test_fourier_amplitudes_single_mode(m0):
    """Sigma = f(r) (1 + eps cos(m0 phi - phi0)) gives A_m0 = eps / 2 in the continuum
    (within the grid's quadrature error).  The quarter-turn images of a column cancel every
    mode m whose parity differs from m0's (and that is not a multiple of 4, which the
    axisymmetric part feeds through the grid's anisotropy) to round-off."""
    from oracle import disk
    n, h = 256, 1.0 / 256
    c = (np.arange(n) + 0.5 - 0.5 * n) * h
    y, x = np.meshgrid(c, c, indexing="ij")
    r = np.sqrt(x * x + y * y)
    eps, phi0 = 0.1, 0.3
    sigma = np.exp(-r / 0.125) * (1.0 + eps * np.cos(m0 * np.arctan2(y, x) - phi0))
    rho = np.stack([sigma / h, sigma * 0.0 + 1e-12])  # two cells per column
    a = disk.fourier_amplitudes(rho, h, 0.25, 8)
    assert abs(a[m0 - 1] - eps / 2) <= 0.01 * eps / 2, a
    for m in range(1, 9):
        if (m - m0) % 2 and m % 4:
            assert a[m - 1] < 1e-13, (m, a)


def _inflow_run(n, bc_lo):
    """1D gas at rest (rho = 1, p = 1, gamma = 1.4) on [0, 1] with a supersonic inflow
    (rho = 1, u = 3, p = 1) prescribed in the ghost cells left of x = 0, run to t = 0.3."""
    z = np.zeros(n)
    u = [a[None, None, :] for a in (np.ones(n), z, z, z, np.full(n, 2.5), np.full(n, 2.5))]
    g = oracle.Grid((n, 1, 1), (1.0 / n, 1.0, 1.0), 1.4, (bc_lo, 0, 0, 0, 0, 0), 0.4,
                    rho_mean=1.0, inflow={0: (1.0, 3.0, 0.0, 0.0, 7.0, 2.5)})
    out, t, steps, dg = oracle.run(g, u, 0.3)
    edges = np.arange(n + 1) / n
    ex = exact.riemann_cell_averages(1.0, 3.0, 1.0, 1.0, 0.0, 1.0, 1.4, 0.0, t, edges, sub=8)
    return float(np.mean(np.abs(out[0].ravel() - ex[0]))), t, dg


def test_inflow_boundary_converges_to_exact_riemann_solution():
    """Inflow boundary: both waves of the Riemann problem (inflow state | gas at rest) move
    right (shocks at 0.61 and 2.39), so on x > 0 the exact solution is the Riemann
    solution with its jump at x = 0.  L1(rho) falls at first order (0.0197, 0.0100,
    0.0046 at 100, 200, 400 cells in the first run; bound 6e-3 at 400), the mass gained
    tends to the inflow rho u t = 0.9 (deficit halving per refinement), and the same
    run with an outflow face stays at rest, far from the exact solution."""
    e1, _, d1 = _inflow_run(100, oracle.BC_INFLOW)
    e2, t, d2 = _inflow_run(200, oracle.BC_INFLOW)
    e4, _, d4 = _inflow_run(400, oracle.BC_INFLOW)
    assert e2 < 0.7 * e1 and e4 < 0.7 * e2 and e4 < 6e-3
    assert all(d["n_nonphys"] == 0 for d in (d1, d2, d4))
    m_exact = 1.0 + 3.0 * t
    gap2, gap4 = m_exact - d2["sums"][0], m_exact - d4["sums"][0]
    assert 0.0 < gap4 < 0.6 * gap2 and gap4 < 4e-3
    e_out, _, _ = _inflow_run(200, oracle.BC_OUTFLOW)
    assert e_out > 0.5


def test_inflow_face_needs_a_state():
    g = oracle.Grid((8, 1, 1), (0.125, 1.0, 1.0), 1.4, (oracle.BC_INFLOW,) + (0,) * 5)
    with pytest.raises(ValueError):
        g.desc()


def _inflow_line(n, ax):
    """The supersonic-inflow problem on a line along axis ax (inflow on its low face, the
    stream's momentum in component ax)."""
    nn = [1, 1, 1]
    nn[ax] = n
    shape = (nn[2], nn[1], nn[0])
    z = np.zeros(shape)
    u = [np.ones(shape), z, z, z, np.full(shape, 2.5), np.full(shape, 2.5)]
    h = [1.0, 1.0, 1.0]
    h[ax] = 1.0 / n
    bc = [oracle.BC_OUTFLOW] * 6
    bc[2 * ax] = oracle.BC_INFLOW
    state = [1.0, 0.0, 0.0, 0.0, 7.0, 2.5]
    state[1 + ax] = 3.0
    g = oracle.Grid(tuple(nn), tuple(h), 1.4, tuple(bc), 0.4, rho_mean=1.0,
                    inflow={2 * ax: tuple(state)})
    out, t, steps, dg = oracle.run(g, u, 0.3)
    return out[0].ravel(), out[1 + ax].ravel(), steps


@pytest.mark.parametrize("ax", [1, 2])
def test_inflow_same_along_every_axis(ax):
    """The inflow problem along y (face 2, m_y) and z (face 4, m_z) gives the x run's
    density and momentum profiles bit for bit, with the same steps: the face index and the
    momentum component of an inflow state follow the axis."""
    r0, m0, s0 = _inflow_line(200, 0)
    r, m, s = _inflow_line(200, ax)
    assert s == s0
    assert np.array_equal(r, r0) and np.array_equal(m, m0)
