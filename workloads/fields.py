"""Initial scalar fields: a Gaussian blob plus seeded uniform noise."""
import numpy as np

from .rng import uniform01


def gaussian_blob(nx, ny, nz, center, sigma, noise_amp, seed, dtype=np.float64):
    """q[k, j, i] = exp(-|(i, j, k) - center|^2 / (2 sigma^2)) + noise_amp * (2u - 1).

    Cell centres sit at integer indices, the blob is not wrapped, and u is the
    uniform draw whose counter is the linear cell index (k*ny + j)*nx + i.
    Returned in x-fastest layout, shape (nz, ny, nx); built one level at a
    time so the largest workloads need no full-size temporaries.
    """
    ci, cj, ck = center
    i = np.arange(nx, dtype=np.float64)
    j = np.arange(ny, dtype=np.float64)
    rij = (j[:, None] - cj) ** 2 + (i[None, :] - ci) ** 2
    q = np.empty((nz, ny, nx), dtype=dtype)
    plane = np.arange(nx * ny, dtype=np.uint64).reshape(ny, nx)
    for k in range(nz):
        lev = np.exp(-(rij + (k - ck) ** 2) / (2.0 * sigma * sigma))
        if noise_amp:
            lev += noise_amp * (2.0 * uniform01(seed, plane + np.uint64(k * nx * ny)) - 1.0)
        q[k] = lev
    return q
