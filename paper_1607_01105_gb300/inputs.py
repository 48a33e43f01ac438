"""Seeded synthetic initial states shaped like the paper's test problems.

This module holds no arithmetic of the PPML scheme: it only builds primitive fields
(rho, v, p) from the problem statements and converts them to the conserved state
(rho, m = rho v, rho E = p/(gamma-1) + rho |v|^2/2, rho eps = p/(gamma-1)) of the
ideal-gas equation of state p = (gamma - 1) rho eps.  Both the oracle tests and the
GPU path take their inputs from here.  Every array is float64, shape (nz, ny, nx).

Problems (all seeded, no external data):
* ``sod_1d``            -- Table 2 shock tubes (row 1 = Sod), 1D.
* ``planar_sod_3d``     -- Sod states split on the plane x = 0.5, uniform in y and z.
* ``point_blast_3d``    -- Sedov-type point blast: rho = 1, p = 1e-5, energy E added as
                           internal energy to the 8 cells touching the centre.
* ``batched_riemann``   -- many independent 1D Riemann problems of uneven lengths.
* ``galactic_disk``     -- exponential, sech^2-thin gas disk in a fixed pseudo-isothermal
                           halo (rho_DM = rho0 / (1 + (r/r0)^2)), perturbed by 1% noise.
* ``advected_wave``, ``aksenov``, ``uniform_flow``, ``vacuum_sphere``, ``random_smooth``
  -- verification states.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

OUTFLOW, PERIODIC, REFLECT = 0, 1, 2
SEED = 1607


@dataclass
class Problem:
    name: str
    n: tuple          # (nx, ny, nz)
    h: tuple          # (hx, hy, hz)
    x0: tuple         # lower corner
    gamma: float
    cfl: float
    bc: tuple         # -x,+x,-y,+y,-z,+z
    t_end: float
    u: list           # six float64 arrays (rho, mx, my, mz, rhoE, rhoeps), shape (nz, ny, nx)
    extra: dict = field(default_factory=dict)

    @property
    def cells(self) -> int:
        return int(self.n[0]) * int(self.n[1]) * int(self.n[2])


def conserved(rho, vx, vy, vz, p, gamma):
    rho = np.asarray(rho, dtype=np.float64)
    shape = rho.shape
    vx = np.broadcast_to(np.asarray(vx, dtype=np.float64), shape)
    vy = np.broadcast_to(np.asarray(vy, dtype=np.float64), shape)
    vz = np.broadcast_to(np.asarray(vz, dtype=np.float64), shape)
    p = np.broadcast_to(np.asarray(p, dtype=np.float64), shape)
    ei = p / (gamma - 1.0)
    en = ei + 0.5 * rho * (vx * vx + vy * vy + vz * vz)
    return [np.ascontiguousarray(a) for a in (rho, rho * vx, rho * vy, rho * vz, en, ei)]


def _centres(n, h, x0):
    return x0 + (np.arange(n) + 0.5) * h


SOD_TABLE2 = {  # paper Table 2: rho_L, v_L, p_L, rho_R, v_R, p_R, x0, t
    1: (1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 0.5, 0.2),
    2: (1.0, -2.0, 0.4, 1.0, 2.0, 0.4, 0.5, 0.15),
    3: (1.0, 0.0, 1000.0, 1.0, 0.0, 0.01, 0.5, 0.012),
}


def sod_1d(n=256, row=1, gamma=1.4, cfl=0.4) -> Problem:
    rl, ul, pl, rr, ur, pr, xs, t = SOD_TABLE2[row]
    h = 1.0 / n
    x = _centres(n, h, 0.0)
    left = x < xs
    rho = np.where(left, rl, rr)[None, None, :]
    vx = np.where(left, ul, ur)[None, None, :]
    p = np.where(left, pl, pr)[None, None, :]
    return Problem(f"sod{row}_1d_{n}", (n, 1, 1), (h, 1.0, 1.0), (0.0, 0.0, 0.0), gamma, cfl,
                   (OUTFLOW,) * 6, t, conserved(rho, vx, 0.0, 0.0, p, gamma),
                   {"states": (rl, ul, pl, rr, ur, pr), "x_split": xs})


def two_blast_waves(n=2400, gamma=1.4, cfl=0.4, t_end=0.038) -> Problem:
    """Two interacting blast waves on [0, 1] (Sec. 'Two Interacting Blast Waves'): rho = 1,
    v = 0, p = 1000 / 0.01 / 100 split at x = 0.1 and 0.9, reflecting walls, 2400 cells.
    The paper shows the result without its time; t_end is the time of the original test."""
    h = 1.0 / n
    x = _centres(n, h, 0.0)
    p = np.where(x < 0.1, 1000.0, np.where(x < 0.9, 0.01, 100.0))[None, None, :]
    rho = np.ones_like(p)
    return Problem(f"two_blast_waves_{n}", (n, 1, 1), (h, 1.0, 1.0), (0.0, 0.0, 0.0), gamma, cfl,
                   (REFLECT, REFLECT, OUTFLOW, OUTFLOW, OUTFLOW, OUTFLOW), t_end, conserved(rho, 0.0, 0.0, 0.0, p, gamma), {})


def planar_sod_3d(n=128, gamma=1.4, cfl=0.2) -> Problem:
    rl, ul, pl, rr, ur, pr, xs, t = SOD_TABLE2[1]
    h = 1.0 / n
    x = _centres(n, h, 0.0)
    left = np.broadcast_to((x < xs)[None, None, :], (n, n, n))
    rho = np.where(left, rl, rr)
    p = np.where(left, pl, pr)
    return Problem(f"planar_sod_3d_{n}", (n, n, n), (h, h, h), (0.0, 0.0, 0.0), gamma, cfl,
                   (OUTFLOW, OUTFLOW, PERIODIC, PERIODIC, PERIODIC, PERIODIC), t,
                   conserved(rho, 0.0, 0.0, 0.0, p, gamma),
                   {"states": (rl, ul, pl, rr, ur, pr), "x_split": xs})


def point_blast_3d(n=256, gamma=5.0 / 3.0, cfl=0.2, energy=1.0, p0=1e-5, rho0=1.0,
                   radius_end=0.4, xi0=1.15) -> Problem:
    """Point blast on [-0.5, 0.5]^3 (n even): E added to the 8 cells touching the origin.
    t_end: time at which R(t) = xi0 (E t^2/rho0)^(1/5) reaches radius_end."""
    if n % 2:
        raise ValueError("n must be even so that 8 cells touch the centre")
    h = 1.0 / n
    rho = np.full((n, n, n), rho0)
    p = np.full((n, n, n), p0)
    u = conserved(rho, 0.0, 0.0, 0.0, p, gamma)
    c = n // 2
    add = energy / (8.0 * h ** 3)
    for f in (4, 5):
        u[f][c - 1:c + 1, c - 1:c + 1, c - 1:c + 1] += add
    t_end = math.sqrt((radius_end / xi0) ** 5 * rho0 / energy)
    return Problem(f"point_blast_3d_{n}", (n, n, n), (h, h, h), (-0.5, -0.5, -0.5), gamma, cfl,
                   (OUTFLOW,) * 6, t_end, u, {"energy": energy, "rho0": rho0})


def advected_wave(n=128, amp=0.2, u0=1.0, p0=1.0, gamma=1.4, cfl=0.4) -> Problem:
    h = 1.0 / n
    edges = np.arange(n + 1) * h
    k = 2.0 * math.pi
    rho = 1.0 + amp * (np.cos(k * edges[:-1]) - np.cos(k * edges[1:])) / (k * h)
    return Problem(f"advected_wave_{n}", (n, 1, 1), (h, 1.0, 1.0), (0.0, 0.0, 0.0), gamma, cfl,
                   (PERIODIC, PERIODIC, OUTFLOW, OUTFLOW, OUTFLOW, OUTFLOW), 1.0 / u0,
                   conserved(rho[None, None, :], u0, 0.0, 0.0, p0, gamma),
                   {"edges": edges, "u0": u0, "amp": amp})


def aksenov(n=628, cfl=0.4, t_end=math.pi / 2.0) -> Problem:
    """Aksenov test on [0, 2 pi], periodic, u = 0, rho = 1 + cos(x)/2 (cell averages),
    gamma = 3 with p = rho^3/3 (so rho eps = rho^3/6 pointwise; the cell average of
    rho^3 is used)."""
    L = 2.0 * math.pi
    h = L / n
    edges = np.arange(n + 1) * h
    xg, wg = np.polynomial.legendre.leggauss(8)
    xs = 0.5 * (edges[:-1, None] + edges[1:, None]) + 0.5 * h * xg
    r = 1.0 + 0.5 * np.cos(xs)
    rho = (0.5 * wg * r).sum(axis=1)
    p = (0.5 * wg * r ** 3 / 3.0).sum(axis=1)
    return Problem(f"aksenov_{n}", (n, 1, 1), (h, 1.0, 1.0), (0.0, 0.0, 0.0), 3.0, cfl,
                   (PERIODIC, PERIODIC, OUTFLOW, OUTFLOW, OUTFLOW, OUTFLOW), t_end,
                   conserved(rho[None, None, :], 0.0, 0.0, 0.0, p[None, None, :], 3.0),
                   {"edges": edges})


def uniform_flow(n=(16, 12, 10), v=(0.7, -0.3, 0.45), rho=1.3, p=0.8, gamma=1.4, cfl=0.2,
                 bc=(PERIODIC,) * 6) -> Problem:
    nx, ny, nz = n
    h = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    r = np.full((nz, ny, nx), rho)
    return Problem("uniform_flow", n, h, (0.0, 0.0, 0.0), gamma, cfl, bc, 1.0,
                   conserved(r, v[0], v[1], v[2], p, gamma))


def random_smooth(n=(24, 20, 16), seed=SEED, gamma=1.4, cfl=0.2, bc=(PERIODIC,) * 6,
                  amp=0.3, modes=3) -> Problem:
    """Sum of a few random periodic Fourier modes in every primitive field."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = n
    h = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    z, y, x = np.meshgrid(_centres(nz, h[2], 0.0), _centres(ny, h[1], 0.0),
                          _centres(nx, h[0], 0.0), indexing="ij")

    def field(base, scale):
        f = np.full((nz, ny, nx), base)
        for _ in range(modes):
            kx, ky, kz = rng.integers(-2, 3, size=3)
            ph = rng.uniform(0, 2 * math.pi)
            f = f + scale * rng.uniform(-1, 1) * np.sin(2 * math.pi * (kx * x + ky * y + kz * z) + ph)
        return f

    rho = field(1.0, amp / modes)
    p = field(1.0, amp / modes)
    vx, vy, vz = field(0.0, 0.5), field(0.0, 0.5), field(0.0, 0.5)
    return Problem("random_smooth", n, h, (0.0, 0.0, 0.0), gamma, cfl, bc, 1.0,
                   conserved(rho, vx, vy, vz, p, gamma))


def random_rough(n=(24, 20, 16), seed=SEED, gamma=1.4, cfl=0.2, bc=(OUTFLOW,) * 6) -> Problem:
    """Cell-wise random positive density/pressure and random velocities (stress test of
    every limiter branch)."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = n
    h = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    shape = (nz, ny, nx)
    rho = np.exp(rng.uniform(np.log(0.2), np.log(5.0), shape))
    p = np.exp(rng.uniform(np.log(0.1), np.log(10.0), shape))
    v = [rng.uniform(-1.0, 1.0, shape) for _ in range(3)]
    return Problem("random_rough", n, h, (0.0, 0.0, 0.0), gamma, cfl, bc, 1.0,
                   conserved(rho, v[0], v[1], v[2], p, gamma))


def vacuum_sphere(n=32, gamma=1.4, cfl=0.2, rho_vac=1e-8, p_vac=1e-8) -> Problem:
    """Gas sphere of unit radius on [-2, 2]^3 (p = rho = 1 inside) in near-vacuum."""
    h = 4.0 / n
    c = _centres(n, h, -2.0)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(x * x + y * y + z * z)
    inside = r <= 1.0
    rho = np.where(inside, 1.0, rho_vac)
    p = np.where(inside, 1.0, p_vac)
    return Problem(f"vacuum_sphere_{n}", (n, n, n), (h, h, h), (-2.0, -2.0, -2.0), gamma, cfl,
                   (OUTFLOW,) * 6, 0.5, conserved(rho, 0.0, 0.0, 0.0, p, gamma))


@dataclass
class Batch:
    """Independent 1D Riemann problems, instance i on [0, 1] with n_i cells."""
    ncells: np.ndarray        # int32 [B]
    h: np.ndarray             # float64 [B]
    t_end: np.ndarray         # float64 [B]
    states: np.ndarray        # float64 [B, 6] rho_L, u_L, p_L, rho_R, u_R, p_R
    offsets: np.ndarray       # int64 [B+1] start of each instance in the packed arrays
    u: list                   # four packed float64 arrays: rho, m, rho E, rho eps
    gamma: float = 1.4
    cfl: float = 0.4
    resampled: int = 0

    @property
    def cells(self) -> int:
        return int(self.offsets[-1])


def batched_riemann(n_inst=512, n_min=128, n_max=4096, seed=SEED, gamma=1.4, cfl=0.4,
                    max_speed=None) -> Batch:
    """Seeded uneven 1D Riemann problems: n_i even in [n_min, n_max], rho ~ U[0.1, 10],
    p = 10^U[-2, 2], u ~ U[-2, 2], split at x = 0.5.  Draws whose exact solution contains
    vacuum are redrawn.  t_end_i = 0.8 * 0.5 / S_max,i with S_max,i the largest exact wave
    speed (given by the max_speed callable), so no wave leaves the domain."""
    rng = np.random.default_rng(seed)
    n = 2 * rng.integers(n_min // 2, n_max // 2 + 1, size=n_inst)
    states = np.zeros((n_inst, 6))
    t_end = np.zeros(n_inst)
    resampled = 0
    for i in range(n_inst):
        while True:
            rl, rr = rng.uniform(0.1, 10.0, 2)
            pl, pr = 10.0 ** rng.uniform(-2.0, 2.0, 2)
            ul, ur = rng.uniform(-2.0, 2.0, 2)
            cl, cr = math.sqrt(gamma * pl / rl), math.sqrt(gamma * pr / rr)
            if ur - ul < 2.0 * (cl + cr) / (gamma - 1.0):
                break
            resampled += 1
        states[i] = (rl, ul, pl, rr, ur, pr)
        smax = max_speed(rl, ul, pl, rr, ur, pr, gamma) if max_speed else \
            max(abs(ul) + cl, abs(ur) + cr) * 2.0
        t_end[i] = 0.8 * 0.5 / smax
    offsets = np.zeros(n_inst + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(n)
    tot = int(offsets[-1])
    rho = np.empty(tot)
    vx = np.empty(tot)
    p = np.empty(tot)
    for i in range(n_inst):
        ni = int(n[i])
        x = (np.arange(ni) + 0.5) / ni
        left = x < 0.5
        rl, ul, pl, rr, ur, pr = states[i]
        sl = slice(offsets[i], offsets[i + 1])
        rho[sl] = np.where(left, rl, rr)
        vx[sl] = np.where(left, ul, ur)
        p[sl] = np.where(left, pl, pr)
    ei = p / (gamma - 1.0)
    u = [rho, rho * vx, ei + 0.5 * rho * vx * vx, ei]
    return Batch(n.astype(np.int32), 1.0 / n.astype(np.float64), t_end, states, offsets,
                 [np.ascontiguousarray(a) for a in u], gamma, cfl, resampled)


def galactic_disk(n=512, gamma=5.0 / 3.0, cfl=0.2, seed=SEED, r0=0.05, rd=0.125,
                  q_toomre=0.8, pert=0.01, floor=1e-6) -> Problem:
    """Gas disk in the plane z = 0 of [-0.5, 0.5]^3 with G = 1.

    Halo (fixed, analytic): rho_DM = rho0 / (1 + (r/r0)^2), potential
    Phi_h = 4 pi G rho0 r0^2 [ ln(1 + x^2)/2 + arctan(x)/x ], x = r/r0, with rho0 set so
    that the halo circular speed at R = rd is 1.  Disk: Sigma = Sigma0 exp(-R/rd),
    rho = Sigma/(2 z0) sech^2(z/z0), z0 = 2h.  Isothermal-like sound speed chosen so that
    Toomre Q = c_s kappa / (pi G Sigma) = q_toomre at R = 2 rd.  Rotation: v_phi^2 =
    R dPhi_h/dR + (R/rho) dp/dR (halo only; self-gravity is added by the caller's Poisson
    solve).  Density floor floor*max(rho) at rest; 1% seeded Gaussian perturbation.
    Returns the state and, in extra, the halo potential array."""
    rng = np.random.default_rng(seed)
    h = 1.0 / n
    c = _centres(n, h, -0.5)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    R = np.sqrt(x * x + y * y)
    r = np.sqrt(R * R + z * z)

    def halo_phi(rr):
        xx = np.maximum(rr / r0, 1e-12)
        return 4.0 * math.pi * rho0 * r0 ** 2 * (0.5 * np.log1p(xx * xx) + np.arctan(xx) / xx)

    def halo_vc2(rr):
        # v_c^2 = G M(<r)/r = 4 pi G rho0 r0^2 (1 - arctan(x)/x)
        xx = np.maximum(rr / r0, 1e-12)
        return 4.0 * math.pi * rho0 * r0 ** 2 * (1.0 - np.arctan(xx) / xx)

    rho0 = 1.0
    rho0 = 1.0 / float(halo_vc2(np.array(rd)))  # v_c(rd) = 1
    z0 = 2.0 * h
    sigma0 = 1.0
    sigma = sigma0 * np.exp(-R / rd)
    rho = sigma / (2.0 * z0) / np.cosh(z / z0) ** 2
    # kappa at R = 2 rd from Omega^2 = v_c^2 / R^2 (halo)
    Rq = 2.0 * rd
    dR = 1e-4
    om2 = lambda RR: float(halo_vc2(np.array(RR))) / RR ** 2
    d_r2om = ((Rq + dR) ** 2 * math.sqrt(om2(Rq + dR)) - (Rq - dR) ** 2 * math.sqrt(om2(Rq - dR))) / (2 * dR)
    kappa = math.sqrt(2.0 * math.sqrt(om2(Rq)) / Rq * d_r2om)
    cs = q_toomre * math.pi * sigma0 * math.exp(-Rq / rd) / kappa
    p = rho * cs * cs / gamma
    rmax = rho.max()
    rho = np.maximum(rho, floor * rmax)
    p = np.maximum(p, floor * rmax * cs * cs / gamma)
    # rotation: v_phi^2 = R dPhi/dR + (R/rho) dp/dR   (dp/dR = (cs^2/gamma) d rho/dR in the disk)
    dlnsig = -1.0 / rd
    vphi2 = halo_vc2(R) + (cs * cs / gamma) * R * dlnsig * (rho > floor * rmax * 1.0001)
    vphi = np.sqrt(np.maximum(vphi2, 0.0))
    inside = rho > floor * rmax * 1.0001
    vphi = np.where(inside, vphi, 0.0)
    Rs = np.maximum(R, 1e-12)
    vx = -vphi * y / Rs
    vy = vphi * x / Rs
    rho = rho * (1.0 + pert * rng.standard_normal(rho.shape) * inside)
    rho = np.maximum(rho, floor * rmax)
    u = conserved(rho, vx, vy, 0.0, p, gamma)
    om = math.sqrt(om2(Rq))
    t_orb = 2.0 * math.pi / om
    return Problem(f"galactic_disk_{n}", (n, n, n), (h, h, h), (-0.5, -0.5, -0.5), gamma, cfl,
                   (OUTFLOW,) * 6, 5.0 * t_orb, u,
                   {"phi_halo": halo_phi(r), "cs": cs, "t_orb": t_orb, "rho0_halo": rho0})
