"""FP64 CPU oracle of the Poisson solves (paper Sec. 'The Poisson solver').

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  The 27-point discretisation of
Delta Phi = 4 pi G rho (eq. stencil27point) is solved on a periodic grid in harmonic space
(the paper's Stages 2-3): sigma = FFT(rho), phi = -(2/3) pi G h^2 sigma /
(1 - prod_a (1 - (2/3) sin^2(pi k_a / N_a))), Phi = inverse FFT(phi).  Reading (G12): the
paper prints the harmonic formula without its minus sign (the stencil's symbol is
-6 (1 - prod_a(...)), negative for k != 0); the k = 0 mode is undefined and set to zero
(the solve is for rho minus its mean); the multipole boundary of the isolated problem is
not combined with the periodic transform.

The isolated solve (``solve_isolated``) follows the paper's three stages with the readings
that make them consistent with each other:
- Stage 1: boundary values of Phi on the shell of cells just outside the grid from the
  monopole and quadrupole of the mass distribution about the coordinate centre, with the
  factor 1/2 of MacCullagh's formula, Phi_b = -G M / r - (G/2)(I_x + I_y + I_z - 3 I_0) / r^3
  (the paper prints the quadrupole term without the 1/2; the two-mass closed form pins it);
  the shell values that enter the stencil of a boundary cell move to the right-hand side.
- Stages 2-3: with Dirichlet data on the shell the operator is diagonal in the sine basis
  sin(pi j (i+1) / (N+1)), j = 1..N (the discrete sine transform of type I, a library
  primitive here), not in the exponential basis the paper prints; the harmonic amplitude is
  the paper's formula with pi j / N replaced by pi j / (2 (N + 1)).
- Right-hand side: 4 pi G h^2 (rho + Delta_7 rho / 12), Delta_7 the 7-point second difference
  with rho = 0 outside the grid.  The paper prints 4 pi G h^2 rho, for which the 27-point
  operator (= h^2 (Delta + h^2 Delta^2 / 12) + O(h^6)) is second-order accurate; the paper
  states fourth order and its Table 1 drops the error 16x per doubling, which this compact
  correction gives.  ``printed_rhs=True`` solves with the right-hand side as printed.
Geometry: cell (i, j, k) of an (nz, ny, nx) array has its centre at
((i + 1/2 - nx/2) h, (j + 1/2 - ny/2) h, (k + 1/2 - nz/2) h): the grid is centred on the
coordinate origin, the centre of the expansion.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.fft

# eq. stencil27point: centre, face, edge and corner weights of h^2 Delta
STENCIL_27 = {"centre": -38.0 / 9.0, "face": 4.0 / 9.0, "edge": 1.0 / 9.0, "corner": 1.0 / 36.0}


def solve_periodic(rho, h, G=1.0):
    """Potential of rho (shape (nz, ny, nx), x fastest) with the 27-point stencil, periodic."""
    rho = np.asarray(rho, dtype=np.float64)
    nz, ny, nx = rho.shape
    sigma = np.fft.rfftn(rho)
    s = []
    for n, m in ((nz, sigma.shape[0]), (ny, sigma.shape[1]), (nx, sigma.shape[2])):
        k = np.arange(m, dtype=np.float64)
        s.append(1.0 - (2.0 / 3.0) * np.sin(math.pi * k / n) ** 2)
    prod = s[0][:, None, None] * s[1][None, :, None] * s[2][None, None, :]
    den = 1.0 - prod
    den[0, 0, 0] = 1.0
    phik = -(2.0 / 3.0) * math.pi * G * h * h * sigma / den
    phik[0, 0, 0] = 0.0
    return np.fft.irfftn(phik, s=rho.shape, axes=(0, 1, 2))


def apply_stencil(phi):
    """h^2 times the 27-point Laplacian of phi (periodic), with the paper's weights."""
    out = STENCIL_27["centre"] * phi
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                nnz = abs(dx) + abs(dy) + abs(dz)
                if nnz == 0:
                    continue
                w = (STENCIL_27["face"], STENCIL_27["edge"], STENCIL_27["corner"])[nnz - 1]
                out = out + w * np.roll(phi, shift=(dz, dy, dx), axis=(0, 1, 2))
    return out


def cell_centres(n, h):
    """Centres (i + 1/2 - n/2) h of the n cells of one axis (grid centred on the origin)."""
    return (np.arange(n, dtype=np.float64) + 0.5 - 0.5 * n) * h


def multipole_moments(rho, h):
    """(M, I_x, I_y, I_z, I_xy, I_xz, I_yz) of the cell masses m_j = rho_j h^3 about the
    origin (Stage 1 of the isolated solve)."""
    rho = np.asarray(rho, dtype=np.float64)
    nz, ny, nx = rho.shape
    z, y, x = np.meshgrid(cell_centres(nz, h), cell_centres(ny, h), cell_centres(nx, h),
                          indexing="ij")
    m = rho * h ** 3
    return (m.sum(), ((z * z + y * y) * m).sum(), ((x * x + z * z) * m).sum(),
            ((x * x + y * y) * m).sum(), (x * y * m).sum(), (x * z * m).sum(),
            (y * z * m).sum())


def multipole_potential(mom, x, y, z, G=1.0):
    """Monopole + quadrupole potential at points (x, y, z) (MacCullagh's formula)."""
    M, Ix, Iy, Iz, Ixy, Ixz, Iyz = mom
    x, y, z = (np.asarray(a, dtype=np.float64) for a in (x, y, z))
    r2 = x * x + y * y + z * z
    r = np.sqrt(r2)
    I0 = ((x * x * Ix + y * y * Iy + z * z * Iz) - 2.0 * (x * y * Ixy + x * z * Ixz + y * z * Iyz)) / r2
    return -G * M / r - 0.5 * G * (Ix + Iy + Iz - 3.0 * I0) / (r2 * r)


def isolated_rhs(rho, h, G=1.0, printed_rhs=False):
    """Right-hand side of the isolated 27-point problem: the source term with the shell
    values of Stage 1 moved over."""
    rho = np.asarray(rho, dtype=np.float64)
    nz, ny, nx = rho.shape
    if printed_rhs:
        src = rho
    else:
        rp = np.pad(rho, 1)  # rho = 0 outside the grid
        lap7 = (rp[2:, 1:-1, 1:-1] + rp[:-2, 1:-1, 1:-1] + rp[1:-1, 2:, 1:-1] +
                rp[1:-1, :-2, 1:-1] + rp[1:-1, 1:-1, 2:] + rp[1:-1, 1:-1, :-2] - 6.0 * rho)
        src = rho + lap7 / 12.0
    rhs = 4.0 * math.pi * G * h * h * src
    # shell of ghost cells (indices -1 and n on each axis) with the multipole values
    mom = multipole_moments(rho, h)
    gz, gy, gx = np.meshgrid(cell_centres(nz + 2, h), cell_centres(ny + 2, h),
                             cell_centres(nx + 2, h), indexing="ij")
    shell = multipole_potential(mom, gx, gy, gz, G)
    shell[1:-1, 1:-1, 1:-1] = 0.0
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                nnz = abs(dx) + abs(dy) + abs(dz)
                if nnz == 0:
                    continue
                w = (STENCIL_27["face"], STENCIL_27["edge"], STENCIL_27["corner"])[nnz - 1]
                rhs -= w * shell[1 + dz:nz + 1 + dz, 1 + dy:ny + 1 + dy, 1 + dx:nx + 1 + dx]
    return rhs, shell


def solve_isolated(rho, h, G=1.0, printed_rhs=False):
    """Potential of an isolated mass distribution rho (shape (nz, ny, nx)) with the
    27-point stencil, boundary values from the multipole expansion (Stages 1-3)."""
    rhs, _ = isolated_rhs(rho, h, G, printed_rhs)
    nz, ny, nx = rhs.shape
    sigma = scipy.fft.dstn(rhs, type=1)
    s = []
    for n in (nz, ny, nx):
        j = np.arange(1, n + 1, dtype=np.float64)
        s.append(1.0 - (2.0 / 3.0) * np.sin(math.pi * j / (2.0 * (n + 1))) ** 2)
    prod = s[0][:, None, None] * s[1][None, :, None] * s[2][None, None, :]
    # eigenvalue of the 27-point operator on the sine mode: 6 (prod - 1)
    phik = sigma / (6.0 * (prod - 1.0))
    return scipy.fft.idstn(phik, type=1)
