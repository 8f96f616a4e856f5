"""Random permeability fields (C order, x fastest: index = x + nx*(y + ny*z)).

All generators take a numpy Generator seeded with PCG64 and return float64
arrays of shape (nz, ny, nx).
"""
import numpy as np


def iid_log_normal(rng, shape, mean_log10, std_log10):
    """log10 K i.i.d. normal per cell; returns K in m^2."""
    return 10.0 ** rng.normal(mean_log10, std_log10, size=shape)


def gaussian_random_field(rng, shape, corr_cells):
    """Stationary Gaussian field with unit variance.

    White noise is convolved periodically (via FFT) with a separable Gaussian
    kernel whose standard deviation along each axis is corr/sqrt(2) cells;
    the result is standardised to sample mean 0 and standard deviation 1.
    `shape` is (nz, ny, nx); `corr_cells` is (lx, ly, lz).
    """
    nz, ny, nx = shape
    lx, ly, lz = corr_cells
    noise = rng.standard_normal(size=shape)

    def kernel_1d(n, corr):
        d = np.minimum(np.arange(n), n - np.arange(n)).astype(np.float64)
        s = corr / np.sqrt(2.0)
        k = np.exp(-0.5 * (d / s) ** 2)
        return k / k.sum()

    kz = kernel_1d(nz, lz)[:, None, None]
    ky = kernel_1d(ny, ly)[None, :, None]
    kx = kernel_1d(nx, lx)[None, None, :]
    kern = kz * ky * kx
    field = np.real(np.fft.ifftn(np.fft.fftn(noise) * np.fft.fftn(kern)))
    field -= field.mean()
    sd = field.std()
    if sd > 0:
        field /= sd
    return field


def channelised(rng, shape, corr_cells, sand_fraction, k_sand, k_shale):
    """Binary facies: sand where a Gaussian field is at or above its
    (1 - sand_fraction) quantile. Returns (K, is_sand)."""
    f = gaussian_random_field(rng, shape, corr_cells)
    thr = np.quantile(f, 1.0 - sand_fraction)
    sand = f >= thr
    K = np.where(sand, k_sand, k_shale).astype(np.float64)
    return K, sand


def layered(rng, shape, n_layers, top_log10, bottom_log10, std_log10):
    """Layered log10 K: nz is split into n_layers equal layers (layer 0 at the
    bottom, z up); layer means vary linearly from bottom_log10 (bottom layer)
    to top_log10 (top layer); within a layer log10 K is i.i.d. normal."""
    nz, ny, nx = shape
    per = max(1, nz // n_layers)
    layer = np.minimum(np.arange(nz) // per, n_layers - 1)
    if n_layers > 1:
        means = bottom_log10 + (top_log10 - bottom_log10) * layer / (n_layers - 1)
    else:
        means = np.full(nz, 0.5 * (top_log10 + bottom_log10))
    logk = means[:, None, None] + rng.normal(0.0, std_log10, size=shape)
    return 10.0 ** logk
