"""Spatially correlated lognormal k_c arrays (the load array C(i,j))."""
import numpy as np

from .rng import std_normal, subseed


def lognormal_kc(nx, ny, seed, epoch, mu=1.0, smooth_sigma=4.0, half_width=8,
                 kmin=1, kmax=64):
    """k_c(i, j) for one epoch.

    A standard-normal field (draw counter = j*nx + i of the epoch's stream) is
    smoothed by a periodic separable Gaussian kernel (std `smooth_sigma`
    cells, taps -half_width..half_width, normalised), re-standardised to zero
    mean and unit variance, mapped to exp(mu + z), clipped to [kmin, kmax] and
    rounded half up to an integer.  Returned as int32, shape (ny, nx).
    """
    s = subseed(seed, 1000 + epoch)
    z = std_normal(s, np.arange(nx * ny, dtype=np.uint64)).reshape(ny, nx)
    taps = np.arange(-half_width, half_width + 1, dtype=np.float64)
    g = np.exp(-taps ** 2 / (2.0 * smooth_sigma ** 2))
    g /= g.sum()
    sm = np.zeros_like(z)
    for t, wt in zip(taps.astype(int), g):
        sm += wt * np.roll(z, t, axis=1)
    z2 = np.zeros_like(z)
    for t, wt in zip(taps.astype(int), g):
        z2 += wt * np.roll(sm, t, axis=0)
    z2 = (z2 - z2.mean()) / z2.std()
    k = np.clip(np.exp(mu + z2), kmin, kmax)
    return np.floor(k + 0.5).astype(np.int32)
