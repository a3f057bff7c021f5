"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds none of the method's arithmetic: it only draws random
vectors and evaluates the prescribed temperature fields of the benchmark
configurations at given points.  Both the CUDA path's callers (tests, bench)
and the oracle's callers take their inputs from here.

Temperature (spherical-shell benchmark setup, Sec. 8): conductive profile
    T_c(r) = r_b (r - r_t) / (r (r_b - r_t))
plus a degree-l, order-m perturbation
    amp * cos(m phi) * P_l^m(cos theta) * sin(pi (r - r_b) / (r_t - r_b)),
theta the colatitude, phi the longitude, P_l^m the unnormalised associated
Legendre function (without Condon-Shortley phase), e.g. P_3^2(x) = 15 x (1 - x^2).
"""
import math

import numpy as np


def assoc_legendre(l, m, x):
    """Unnormalised associated Legendre function P_l^m(x), no Condon-Shortley phase."""
    x = np.asarray(x, dtype=np.float64)
    pmm = np.ones_like(x)
    somx2 = np.sqrt(np.maximum(0.0, (1.0 - x) * (1.0 + x)))
    fact = 1.0
    for _ in range(m):
        pmm = pmm * fact * somx2
        fact += 2.0
    if l == m:
        return pmm
    pmmp1 = x * (2 * m + 1) * pmm
    if l == m + 1:
        return pmmp1
    pll = None
    for ll in range(m + 2, l + 1):
        pll = (x * (2 * ll - 1) * pmmp1 - (ll + m - 1) * pmm) / (ll - m)
        pmm, pmmp1 = pmmp1, pll
    return pll


def temperature(xyz, r_b, r_t, amp=0.01, l=3, m=2, normalize=False):
    """T at Cartesian points xyz (n, 3) of the shell r_b <= |x| <= r_t."""
    xyz = np.asarray(xyz, dtype=np.float64)
    r = np.sqrt((xyz[:, 0] * xyz[:, 0] + xyz[:, 1] * xyz[:, 1]) + xyz[:, 2] * xyz[:, 2])
    cth = np.clip(xyz[:, 2] / r, -1.0, 1.0)
    phi = np.arctan2(xyz[:, 1], xyz[:, 0])
    ang = np.cos(m * phi) * assoc_legendre(l, m, cth)
    if normalize:
        grid = np.linspace(-1.0, 1.0, 2001)
        ang = ang / np.max(np.abs(assoc_legendre(l, m, grid)))
    Tc = r_b * (r - r_t) / (r * (r_b - r_t))
    return Tc + amp * ang * np.sin(math.pi * (r - r_b) / (r_t - r_b))


def normal(n, seed, scale=1.0):
    """n seeded N(0, scale^2) draws (numpy PCG64)."""
    return np.random.default_rng(seed).normal(0.0, scale, size=n)


def lognormal_viscosity(n, seed, sigma=1.0):
    """n seeded positive viscosities exp(N(0, sigma^2))."""
    return np.exp(np.random.default_rng(seed).normal(0.0, sigma, size=n))
