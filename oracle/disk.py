"""FP64 CPU oracle of the global Fourier amplitudes of a disk (paper Sec. on the
gravitationally unstable disks, eq. of A_m(t)).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  A_m = |sum Sigma e^{i m phi}| / sum Sigma
over the columns whose centre lies within R_f of the axis, Sigma = sum over z of rho times
h (the column density; the cell area cancels), phi the polar angle of the column centre
(atan2(y, x)).  Geometry as in the isolated Poisson solve: cell (i, j, k) is centred at
((i + 1/2 - nx/2) h, (j + 1/2 - ny/2) h, (k + 1/2 - nz/2) h).
"""
from __future__ import annotations

import numpy as np


def fourier_amplitudes(rho, h, r_f, m_max):
    """A_1 .. A_m_max of rho (shape (nz, ny, nx)) over the columns with r <= r_f."""
    rho = np.asarray(rho, dtype=np.float64)
    nz, ny, nx = rho.shape
    sigma = rho.sum(axis=0) * h
    x = (np.arange(nx) + 0.5 - 0.5 * nx) * h
    y = (np.arange(ny) + 0.5 - 0.5 * ny) * h
    Y, X = np.meshgrid(y, x, indexing="ij")
    inside = X * X + Y * Y <= r_f * r_f
    phi = np.arctan2(Y, X)
    total = sigma[inside].sum()
    out = []
    for m in range(1, m_max + 1):
        z = (sigma[inside] * np.exp(1j * m * phi[inside])).sum()
        out.append(abs(z) / total)
    return np.array(out)
