"""Seeded synthetic inputs shared by the CUDA path, the tests and the oracle.

This module holds no arithmetic of the method: only velocity fields and
right-hand sides, generated on the host with NumPy's PCG64 (``default_rng``).
They stand in for the paper's velocity fields and forces (Sec. 3, Sec. 5),
whose formulas are not given in the paper:

* ``random_velocity``: Gaussian-filtered N(0,1) white noise (correlation
  length ``corr`` in domain units, periodic FFT filter), mapped affinely onto
  [lo, hi].
* ``lens_velocity``: a converging Gaussian lens c = 4/3 (1 - 0.5 exp(-32 |x-x0|^2)).
* ``point_sources``: Gaussian point sources exp(-|x-x0|^2/(2 s^2))/(2 pi s^2)
  (unit mass in 2D; (2 pi s^2)^(3/2) in 3D) with s = h, centres uniform in
  [eta, 1-eta]^d.
* ``waveguide_velocity``: a vertical waveguide with Gaussian cross-section,
  c = 4/3 (1 - 0.5 exp(-32 (x1 - 1/2)^2)) (the lens profile in x1 only,
  constant along x2).
* ``wave_packet``: a Gaussian wave packet exp(-|x-x0|^2/(2 w^2))
  exp(i k d.(x-x0)), k = omega / c0, with envelope width w equal to one
  wavelength 2 pi c0 / omega, centred at (0.125, 0.125) and pointing along
  d = (1, 1)/sqrt(2).

Grids are the paper's: n interior points per axis, h = 1/(n+1), arrays
indexed [x_d, ..., x_1] with x_1 fastest.
"""
import numpy as np

__all__ = ["random_velocity", "lens_velocity", "waveguide_velocity", "constant_velocity", "point_sources",
           "centered_source", "wave_packet", "random_rhs", "cnn_init_params"]


def _grid(n):
    h = 1.0 / (n + 1)
    return h, h * np.arange(1, n + 1, dtype=np.float64)


def random_velocity(n, seed, dim=2, corr=0.05, lo=0.8, hi=1.2):
    """Smooth random field in [lo, hi] (float64, shape (n,)*dim)."""
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal((n,) * dim)
    sig = corr * (n + 1)                       # filter std in grid points
    F = np.fft.fftn(noise)
    k2 = np.zeros((n,) * dim)
    for ax in range(dim):
        k = np.fft.fftfreq(n)
        shape = [1] * dim
        shape[ax] = n
        k2 = k2 + (k.reshape(shape) ** 2)
    F *= np.exp(-2.0 * (np.pi ** 2) * (sig ** 2) * k2)
    sm = np.real(np.fft.ifftn(F))
    a, b = sm.min(), sm.max()
    return lo + (hi - lo) * (sm - a) / (b - a)


def lens_velocity(n, dim=2):
    """Converging Gaussian lens centred in the domain."""
    _, x = _grid(n)
    grids = np.meshgrid(*([x] * dim), indexing="ij")
    r2 = sum((g - 0.5) ** 2 for g in grids)
    return (4.0 / 3.0) * (1.0 - 0.5 * np.exp(-32.0 * r2))


def waveguide_velocity(n):
    """Vertical waveguide (2D): the lens profile in x1 only, constant along x2."""
    _, x = _grid(n)
    c1 = (4.0 / 3.0) * (1.0 - 0.5 * np.exp(-32.0 * (x - 0.5) ** 2))
    return np.tile(c1[None, :], (n, 1))


def wave_packet(n, omega, center=(0.125, 0.125), direction=(1.0, 1.0), c0=1.0):
    """Gaussian wave packet (2D, complex128, shape (1, n, n)): envelope of one
    wavelength width at ``center``, plane-wave phase along ``direction``."""
    _, x = _grid(n)
    X2, X1 = np.meshgrid(x, x, indexing="ij")
    k = omega / c0
    w = 2 * np.pi * c0 / omega
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    r1, r2 = X1 - center[0], X2 - center[1]
    f = np.exp(-(r1 ** 2 + r2 ** 2) / (2 * w ** 2)) * np.exp(1j * k * (d[0] * r1 + d[1] * r2))
    return f.astype(np.complex128)[None]


def constant_velocity(n, dim=2, value=1.0):
    return np.full((n,) * dim, value, dtype=np.float64)


def _gaussian_patch(n, center, dim, width):
    """Gaussian of std ``width`` (domain units) sampled on the grid near ``center``."""
    h, x = _grid(n)
    out = np.zeros((n,) * dim, dtype=np.float64)
    rad = int(np.ceil(8 * width / h)) + 1
    sl = []
    coords = []
    # arrays are indexed [x_dim, ..., x_1]; center is (x_1, ..., x_dim)
    for ax in range(dim):
        cx = center[dim - 1 - ax]
        k0 = max(0, int(round(cx / h)) - 1 - rad)
        k1 = min(n, int(round(cx / h)) - 1 + rad + 1)
        sl.append(slice(k0, k1))
        coords.append(x[k0:k1] - cx)
    grids = np.meshgrid(*coords, indexing="ij")
    r2 = sum(g ** 2 for g in grids)
    out[tuple(sl)] = np.exp(-r2 / (2 * width ** 2)) / ((2 * np.pi * width ** 2) ** (dim / 2.0))
    return out


def point_sources(n, nrhs, seed, bp, dim=2):
    """``nrhs`` Gaussian point sources (s = h) at seeded uniform positions in
    [eta, 1-eta]^dim, eta = bp h.  Returns complex128 (nrhs, n, ..., n)."""
    rng = np.random.default_rng(seed)
    h = 1.0 / (n + 1)
    eta = bp * h
    centers = rng.uniform(eta, 1.0 - eta, size=(nrhs, dim))
    f = np.zeros((nrhs,) + (n,) * dim, dtype=np.complex128)
    for r in range(nrhs):
        f[r] = _gaussian_patch(n, centers[r], dim, h)
    return f


def centered_source(n, dim=2, center=None):
    """One Gaussian point source (s = h) at ``center`` (default: domain centre)."""
    h = 1.0 / (n + 1)
    c = (0.5,) * dim if center is None else center
    return _gaussian_patch(n, c, dim, h).astype(np.complex128)[None]


def random_rhs(n, nrhs, seed, dim=2):
    """Dense complex N(0,1) right-hand sides (used by parity tests)."""
    rng = np.random.default_rng(seed)
    shape = (nrhs,) + (n,) * dim
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def cnn_init_params(seed, out_scale=0.1):
    """Initial parameters of the post-correction network (float32, flat layout
    W1[3][3][2][32], b1, W2[3][3][32][32], b2, W3[3][3][32][2], b3): He-normal
    weights (std sqrt(2 / fan_in), fan_in = 9 * input channels), zero biases,
    the last layer scaled by ``out_scale`` so that training starts near the
    plain sweep."""
    rng = np.random.default_rng(seed)
    parts = []
    for cin, cout, scale in ((2, 32, 1.0), (32, 32, 1.0), (32, 2, out_scale)):
        w = rng.standard_normal((3, 3, cin, cout)) * np.sqrt(2.0 / (9 * cin)) * scale
        parts += [w.ravel(), np.zeros(cout)]
    return np.concatenate(parts).astype(np.float32)
