"""Exact unsteady-Stokes step on a periodic grid (FP64, NumPy FFT).

TEST INFRASTRUCTURE: the fluid stand-in that the oracle pins use to close the
two-way coupling loop on small grids.  It advances the linear unsteady Stokes
equations (the disturbance problem of Sec. 2.2 and App. A.5) by one step of
length dt with the forcing, diffusion and projection split of App. A.5:

    u_hat <- exp(-nu |k|^2 dt) P(k) (u_hat + dt S_hat),

P(k) = I - k k^T / |k|^2 the Leray projector (identity on the mean mode).
Fields are [3, nz, ny, nx] with nodes at j L / N.
"""

from __future__ import annotations

import numpy as np


def wavenumbers(n, L):
    nx, ny, nz = n
    kx = 2 * np.pi * np.fft.fftfreq(nx, d=L[0] / nx)
    ky = 2 * np.pi * np.fft.fftfreq(ny, d=L[1] / ny)
    kz = 2 * np.pi * np.fft.fftfreq(nz, d=L[2] / nz)
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    return KX, KY, KZ


def stokes_step(u, S, nu, dt, L):
    """One exact Stokes step of the periodic field u forced by S."""
    n = (u.shape[3], u.shape[2], u.shape[1])
    KX, KY, KZ = wavenumbers(n, L)
    K2 = KX ** 2 + KY ** 2 + KZ ** 2
    uh = np.fft.fftn(u + dt * S, axes=(1, 2, 3))
    K2s = np.where(K2 == 0.0, 1.0, K2)
    kdotu = (KX * uh[0] + KY * uh[1] + KZ * uh[2]) / K2s
    uh[0] -= KX * kdotu
    uh[1] -= KY * kdotu
    uh[2] -= KZ * kdotu
    uh *= np.exp(-nu * K2 * dt)[None]
    return np.real(np.fft.ifftn(uh, axes=(1, 2, 3)))
