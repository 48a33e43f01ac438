"""Exact solutions used to pin the oracle (test infrastructure only).

None of this shares arithmetic with the scheme in ``ppml_oracle.c``; these are the
textbook solutions the paper compares against:

* ``riemann_exact`` -- the exact Riemann problem of the ideal-gas Euler equations (the
  shock tubes of the paper's Table 2): a Newton iteration on the star pressure with the
  shock (Rankine-Hugoniot) and rarefaction (isentropic) branches, then self-similar
  sampling including rarefaction fans.
* ``aksenov_exact`` -- the smooth periodic solution of the Aksenov test (Sec. "The
  Aksenov Test").  The printed EOS p = rho^3 is read as p = rho^3/3 (gamma = 3): only
  then is c = rho, the Riemann invariants u +- rho obey Burgers' equation, and the
  printed rho, u are their half difference and half sum.  The solution is implicit and
  is solved per point by Newton's method.
* ``advected_wave_exact`` -- translation of a density profile in uniform flow with
  constant pressure (an exact solution of the Euler equations).
* ``sedov_xi0`` -- the similarity constant of the Sedov-Taylor blast wave, obtained by
  integrating the self-similar ODEs numerically (no tabulated value is used).
"""
from __future__ import annotations

import math

import numpy as np


# --------------------------------------------------------------------------- Riemann

def _f_and_df(p, rk, pk, ck, g):
    if p > pk:  # shock
        A = 2.0 / ((g + 1.0) * rk)
        B = (g - 1.0) / (g + 1.0) * pk
        s = math.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (B + p))
    # rarefaction
    pr = p / pk
    f = 2.0 * ck / (g - 1.0) * (pr ** ((g - 1.0) / (2.0 * g)) - 1.0)
    df = 1.0 / (rk * ck) * pr ** (-(g + 1.0) / (2.0 * g))
    return f, df


def riemann_star(rl, ul, pl, rr, ur, pr, g):
    """Star-region pressure and velocity of the exact Riemann problem."""
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    if 2.0 * (cl + cr) / (g - 1.0) <= ur - ul:
        raise ValueError("initial data generate vacuum")
    # two-rarefaction guess, then Newton
    z = (g - 1.0) / (2.0 * g)
    p = ((cl + cr - 0.5 * (g - 1.0) * (ur - ul)) / (cl / pl ** z + cr / pr ** z)) ** (1.0 / z)
    p = max(p, 1e-14 * min(pl, pr))
    for _ in range(200):
        fl, dfl = _f_and_df(p, rl, pl, cl, g)
        fr, dfr = _f_and_df(p, rr, pr, cr, g)
        f = fl + fr + (ur - ul)
        pn = p - f / (dfl + dfr)
        if pn <= 0.0:
            pn = 0.5 * p
        if abs(pn - p) <= 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _f_and_df(p, rl, pl, cl, g)
    fr, _ = _f_and_df(p, rr, pr, cr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def riemann_sample(rl, ul, pl, rr, ur, pr, g, s):
    """Exact (rho, u, p) at similarity coordinate s = (x - x0)/t (array)."""
    s = np.asarray(s, dtype=np.float64)
    ps, us = riemann_star(rl, ul, pl, rr, ur, pr, g)
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    gm, gp = g - 1.0, g + 1.0
    rho = np.empty_like(s)
    u = np.empty_like(s)
    p = np.empty_like(s)
    for idx, si in np.ndenumerate(s):
        if si <= us:  # left of contact
            if ps > pl:  # left shock
                SL = ul - cl * math.sqrt(gp / (2 * g) * ps / pl + gm / (2 * g))
                if si <= SL:
                    r, v, q = rl, ul, pl
                else:
                    r = rl * ((ps / pl + gm / gp) / (gm / gp * ps / pl + 1.0))
                    v, q = us, ps
            else:  # left rarefaction
                SH = ul - cl
                cs = cl * (ps / pl) ** (gm / (2 * g))
                ST = us - cs
                if si <= SH:
                    r, v, q = rl, ul, pl
                elif si >= ST:
                    r, v, q = rl * (ps / pl) ** (1.0 / g), us, ps
                else:
                    c = 2.0 / gp * (cl + gm / 2.0 * (ul - si))
                    v = 2.0 / gp * (cl + gm / 2.0 * ul + si)
                    r = rl * (c / cl) ** (2.0 / gm)
                    q = pl * (c / cl) ** (2.0 * g / gm)
        else:  # right of contact
            if ps > pr:
                SR = ur + cr * math.sqrt(gp / (2 * g) * ps / pr + gm / (2 * g))
                if si >= SR:
                    r, v, q = rr, ur, pr
                else:
                    r = rr * ((ps / pr + gm / gp) / (gm / gp * ps / pr + 1.0))
                    v, q = us, ps
            else:
                SH = ur + cr
                cs = cr * (ps / pr) ** (gm / (2 * g))
                ST = us + cs
                if si >= SH:
                    r, v, q = rr, ur, pr
                elif si <= ST:
                    r, v, q = rr * (ps / pr) ** (1.0 / g), us, ps
                else:
                    c = 2.0 / gp * (cr - gm / 2.0 * (ur - si))
                    v = 2.0 / gp * (-cr + gm / 2.0 * ur + si)
                    r = rr * (c / cr) ** (2.0 / gm)
                    q = pr * (c / cr) ** (2.0 * g / gm)
        rho[idx], u[idx], p[idx] = r, v, q
    return rho, u, p


def riemann_max_speed(rl, ul, pl, rr, ur, pr, g):
    """Largest |wave speed| of the exact solution (outermost shock or rarefaction head)."""
    ps, us = riemann_star(rl, ul, pl, rr, ur, pr, g)
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    gm, gp = g - 1.0, g + 1.0
    if ps > pl:
        sl = ul - cl * math.sqrt(gp / (2 * g) * ps / pl + gm / (2 * g))
    else:
        sl = ul - cl
    if ps > pr:
        sr = ur + cr * math.sqrt(gp / (2 * g) * ps / pr + gm / (2 * g))
    else:
        sr = ur + cr
    return max(abs(sl), abs(sr))


def riemann_cell_averages(rl, ul, pl, rr, ur, pr, g, x0, t, edges, sub=64):
    """Cell averages of the exact conserved variables (rho, m, rho E) over cells with the
    given edges, by Gauss-Legendre quadrature of sub points on sub-intervals."""
    edges = np.asarray(edges, dtype=np.float64)
    n = edges.size - 1
    xg, wg = np.polynomial.legendre.leggauss(4)
    out = np.zeros((3, n))
    for i in range(n):
        a, b = edges[i], edges[i + 1]
        sb = np.linspace(a, b, sub + 1)
        xs = (0.5 * (sb[1:, None] + sb[:-1, None]) + 0.5 * (sb[1:, None] - sb[:-1, None]) * xg).ravel()
        ws = (0.5 * (sb[1:, None] - sb[:-1, None]) * wg).ravel()
        r, v, p = riemann_sample(rl, ul, pl, rr, ur, pr, g, (xs - x0) / t)
        E = p / (g - 1.0) + 0.5 * r * v * v
        out[0, i] = np.sum(ws * r) / (b - a)
        out[1, i] = np.sum(ws * r * v) / (b - a)
        out[2, i] = np.sum(ws * E) / (b - a)
    return out


# --------------------------------------------------------------------------- Aksenov

def aksenov_exact(x, t, newton_iters=60):
    """(rho, u) of the Aksenov solution with c = rho (gamma = 3, p = rho^3/3).

    Riemann invariants R+ = u + rho and R- = u - rho are constant along dx/dt = R+ and
    dx/dt = R- and start as R+(x,0) = 1 + cos(x)/2, R-(x,0) = -1 - cos(x)/2.  So
    R+(x,t) = 1 + cos(x - R+ t)/2 and R-(x,t) = -1 - cos(x - R- t)/2, solved by Newton.
    """
    x = np.asarray(x, dtype=np.float64)

    def solve(sign):
        R = sign * (1.0 + 0.5 * np.cos(x))
        for _ in range(newton_iters):
            arg = x - R * t
            F = R - sign * (1.0 + 0.5 * np.cos(arg))
            dF = 1.0 - sign * 0.5 * np.sin(arg) * t
            R = R - F / dF
        return R

    Rp = solve(1.0)
    Rm = solve(-1.0)
    return 0.5 * (Rp - Rm), 0.5 * (Rp + Rm)


def aksenov_cell_averages(edges, t, sub=8):
    """Cell averages of rho and of m = rho u of the Aksenov solution."""
    edges = np.asarray(edges, dtype=np.float64)
    xg, wg = np.polynomial.legendre.leggauss(6)
    a = edges[:-1, None]
    b = edges[1:, None]
    rho = np.zeros(edges.size - 1)
    mom = np.zeros(edges.size - 1)
    for s in range(sub):
        lo = a + (b - a) * s / sub
        hi = a + (b - a) * (s + 1) / sub
        xs = 0.5 * (lo + hi) + 0.5 * (hi - lo) * xg
        r, u = aksenov_exact(xs, t)
        w = 0.5 * (hi - lo) * wg
        rho += np.sum(w * r, axis=1)
        mom += np.sum(w * r * u, axis=1)
    return rho / (b - a)[:, 0], mom / (b - a)[:, 0]


# --------------------------------------------------------------------- advected wave

def advected_wave_exact(edges, t, u0=1.0, amp=0.2, k=2.0 * math.pi, period=1.0):
    """Cell averages of rho = 1 + amp sin(k (x - u0 t)) on a periodic domain (exact)."""
    edges = np.asarray(edges, dtype=np.float64)
    a = edges[:-1] - u0 * t
    b = edges[1:] - u0 * t
    return 1.0 + amp * (np.cos(k * a) - np.cos(k * b)) / (k * (b - a))


# --------------------------------------------------------------------------- Sedov

def sedov_xi0(gamma, n=4000, xi_min=1e-4):
    """Similarity constant xi0 of the 3D point blast, R(t) = xi0 (E t^2 / rho0)^(1/5).

    Self-similar variables (xi = r/R, ' = d/d ln xi, D = dR/dt = 2R/(5t)):
    v = D xi V, rho = rho0 G, c^2 = (D xi)^2 Z.  Continuity, momentum and entropy give
        V' + (V-1) (ln G)'                       = -3 V
        (V-1) V' + (Z/g) (ln G)' + Z'/g          = V (5/2 - V) - 2 Z/g
        -(g-1)(V-1) (ln G)' + (V-1) Z'/Z         = 5 - 2 V
    started from the strong-shock jump at xi = 1 and integrated inward (RK4 in ln xi).
    Energy: E = (16 pi / 25) rho0 R^5 t^-2 int_0^1 G (V^2/2 + Z/(g(g-1))) xi^4 dxi.
    """
    g = float(gamma)

    def rhs(y):
        V, lnG, Z = y
        M = np.array([[1.0, V - 1.0, 0.0],
                      [V - 1.0, Z / g, 1.0 / g],
                      [0.0, -(g - 1.0) * (V - 1.0), (V - 1.0) / Z]])
        b = np.array([-3.0 * V, V * (2.5 - V) - 2.0 * Z / g, 5.0 - 2.0 * V])
        return np.linalg.solve(M, b)

    y = np.array([2.0 / (g + 1.0), math.log((g + 1.0) / (g - 1.0)),
                  2.0 * g * (g - 1.0) / (g + 1.0) ** 2])
    h = math.log(xi_min) / n
    lx = 0.0
    xs, integ = [1.0], []

    def f_of(y, xi):
        V, lnG, Z = y
        return math.exp(lnG) * (0.5 * V * V + Z / (g * (g - 1.0))) * xi ** 4

    integ.append(f_of(y, 1.0))
    for _ in range(n):
        k1 = rhs(y)
        k2 = rhs(y + 0.5 * h * k1)
        k3 = rhs(y + 0.5 * h * k2)
        k4 = rhs(y + h * k3)
        y = y + h / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
        lx += h
        xs.append(math.exp(lx))
        integ.append(f_of(y, math.exp(lx)))
    xs = np.array(xs[::-1])
    integ = np.array(integ[::-1])
    I = np.trapezoid(integ, xs)
    return (16.0 * math.pi / 25.0 * I) ** (-0.2)
