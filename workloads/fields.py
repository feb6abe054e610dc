"""Initial scalar fields: a Gaussian blob plus seeded uniform noise."""
import numpy as np

from .rng import uniform01


def gaussian_blob(nx, ny, nz, center, sigma, noise_amp, seed, dtype=np.float64):
    """q[k, j, i] = exp(-|(i, j, k) - center|^2 / (2 sigma^2)) + noise_amp * (2u - 1).

    Cell centres sit at integer indices, the blob is not wrapped, and u is the
    uniform draw whose counter is the linear cell index (k*ny + j)*nx + i.
    Returned in x-fastest layout, shape (nz, ny, nx).
    """
    ci, cj, ck = center
    i = np.arange(nx, dtype=np.float64)
    j = np.arange(ny, dtype=np.float64)
    k = np.arange(nz, dtype=np.float64)
    r2 = ((k[:, None, None] - ck) ** 2 + (j[None, :, None] - cj) ** 2
          + (i[None, None, :] - ci) ** 2)
    q = np.exp(-r2 / (2.0 * sigma * sigma))
    if noise_amp:
        idx = np.arange(nx * ny * nz, dtype=np.uint64).reshape(nz, ny, nx)
        q += noise_amp * (2.0 * uniform01(seed, idx) - 1.0)
    return q.astype(dtype)
