"""Seeded densities for the synthetic workloads."""
import numpy as np


def _assoc_legendre(n, m, x):
    """P_n^m(x) for m >= 0 without the Condon-Shortley phase (input helper)."""
    pmm = np.ones_like(x)
    s = np.sqrt(np.clip(1 - x * x, 0, None))
    for i in range(1, m + 1):
        pmm = pmm * (2 * i - 1) * s
    if n == m:
        return pmm
    pm1 = x * (2 * m + 1) * pmm
    if n == m + 1:
        return pm1
    for k in range(m + 2, n + 1):
        pm1, pmm = ((2 * k - 1) * x * pm1 - (k + m - 1) * pmm) / (k - m), pm1
    return pm1


def real_sph_harm(n, m, xyz):
    """Real spherical harmonic of degree n, order m at the directions of xyz (N,3):
    cos(m phi) P_n^m for m >= 0, sin(|m| phi) P_n^|m| for m < 0 (unnormalised)."""
    r = np.linalg.norm(xyz, axis=1)
    x = xyz[:, 2] / r
    phi = np.arctan2(xyz[:, 1], xyz[:, 0])
    p = _assoc_legendre(n, abs(m), x)
    return p * (np.cos(m * phi) if m >= 0 else np.sin(-m * phi))


def sphere_density(xyz, rng):
    """1 + 0.5 x y + U(-0.1, 0.1)."""
    return 1.0 + 0.5 * xyz[:, 0] * xyz[:, 1] + rng.uniform(-0.1, 0.1, len(xyz))


def harmonic_density(xyz, rng, n_terms=8, max_degree=6):
    """Sum of n_terms random real spherical harmonics of degree <= max_degree at
    x/|x|, with N(0,1) coefficients (normalised to unit max)."""
    out = np.zeros(len(xyz))
    for _ in range(n_terms):
        n = int(rng.integers(0, max_degree + 1))
        m = int(rng.integers(-n, n + 1))
        f = real_sph_harm(n, m, xyz)
        f = f / max(np.abs(f).max(), 1e-300)
        out += rng.standard_normal() * f
    return out


def plane_wave_density(xyz, k, rng):
    """e^{i k d.x} with a seeded unit direction d (complex128)."""
    d = rng.standard_normal(3)
    d /= np.linalg.norm(d)
    return np.exp(1j * k * (xyz @ d))
