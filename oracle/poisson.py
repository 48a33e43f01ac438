"""FP64 CPU oracle of the periodic Poisson solve (paper Sec. 'The Poisson solver').

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  The 27-point discretisation of
Delta Phi = 4 pi G rho (eq. stencil27point) is solved on a periodic grid in harmonic space
(the paper's Stages 2-3): sigma = FFT(rho), phi = -(2/3) pi G h^2 sigma /
(1 - prod_a (1 - (2/3) sin^2(pi k_a / N_a))), Phi = inverse FFT(phi).  Reading (G12): the
paper prints the harmonic formula without its minus sign (the stencil's symbol is
-6 (1 - prod_a(...)), negative for k != 0); the k = 0 mode is undefined and set to zero
(the solve is for rho minus its mean); the multipole boundary of the isolated problem is
not combined with the periodic transform.
"""
from __future__ import annotations

import math

import numpy as np

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
    return np.fft.irfftn(phik, s=rho.shape)


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
