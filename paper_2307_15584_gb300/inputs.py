"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module only draws random numbers; it holds none of the QMC method's
arithmetic.  Random quantities the method consumes (initial Sobol' direction
numbers, scramble seeds, lattice generator words, Cranley-Patterson shifts,
integrand parameters, per-integral sample counts) are produced here and passed
to both the CUDA path and the oracle as plain arrays.

All draws come from splitmix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: word(key, k) = mix64(key + (k + 1) * 0x9E3779B97F4A7C15).
"""
from __future__ import annotations

import math

import numpy as np

DEFAULT_SEED = 20230728

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def words64(key, counters) -> np.ndarray:
    """splitmix64 output number `counters` of the stream seeded with `key`."""
    key = np.asarray(key, dtype=np.uint64)
    k = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(key + (k + np.uint64(1)) * _GOLDEN)


def words32(key, counters) -> np.ndarray:
    return (words64(key, counters) >> np.uint64(32)).astype(np.uint32)


def uniform01(key, counters) -> np.ndarray:
    """Doubles in [0,1) from the top 53 bits."""
    return (words64(key, counters) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _key(seed: int, tag: int) -> np.uint64:
    return words64(np.uint64(seed), np.uint64(tag))


# stream tags (distinct streams per purpose)
_T_DIRECTION, _T_SCRAMBLE, _T_LATTICE_G, _T_LATTICE_SHIFT = 1, 2, 3, 4
_T_GENZ, _T_THETA, _T_COUNTS, _T_PIXEL, _T_TARGET = 5, 6, 7, 8, 9
_T_IMAGE = 10


def sobol_raw_init(s: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """Raw random words [s][7] seeding the initial direction numbers m_k, k <= 7."""
    return words32(_key(seed, _T_DIRECTION), np.arange(7 * s)).reshape(s, 7)


def scramble_seeds(s: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """One 32-bit seed per dimension [s]."""
    return words32(_key(seed, _T_SCRAMBLE), np.arange(s))


def pixel_seeds(n: int, s: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """Per-integral seeds [n][s]: word j of the stream keyed by word p of the pixel stream."""
    base = words64(_key(seed, _T_PIXEL), np.arange(n, dtype=np.uint64))
    j = np.arange(s, dtype=np.uint64)
    return words32(base[:, None], j[None, :])


def lattice_generator(s: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """Raw generator words [s] (the lattice forces each one odd)."""
    return words32(_key(seed, _T_LATTICE_G), np.arange(s))


def lattice_shift(s: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """Cranley-Patterson shifts [s] in units of 2^-32."""
    return words32(_key(seed, _T_LATTICE_SHIFT), np.arange(s))


def genz_params(family: str, s: int, index: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """fp32 [2s] = (a[s], u[s]); a ~ U[1,5] (product peak) or U[0,1] (oscillatory), u ~ U[0,1]."""
    tag = {"product_peak": 0, "oscillatory": 1}[family]
    key = words64(_key(seed, _T_GENZ), np.uint64(tag * 1000 + index))
    r = uniform01(key, np.arange(2 * s))
    a = 1.0 + 4.0 * r[:s] if family == "product_peak" else r[:s]
    return np.concatenate([a, r[s:]]).astype(np.float32)


def gaussmix_theta(n: int, seed: int = DEFAULT_SEED, tag: int = _T_THETA) -> np.ndarray:
    """fp32 [n][16]: per component (w ~ U[0,1], mu ~ U[0,1], nu ~ U[0,1], sigma ~ U[0.05,0.3])."""
    r = uniform01(_key(seed, tag), np.arange(16 * n, dtype=np.uint64)).reshape(n, 4, 4)
    r[:, :, 3] = 0.05 + 0.25 * r[:, :, 3]
    return r.reshape(n, 16).astype(np.float32)


def log_uniform_counts(n: int, lo: int = 1, hi: int = 65536, seed: int = DEFAULT_SEED) -> np.ndarray:
    """u32 [n]: clamp(floor(exp(U ln hi)), lo, hi), U ~ U[0,1) -- log-uniform sample counts."""
    u = uniform01(_key(seed, _T_COUNTS), np.arange(n, dtype=np.uint64))
    c = np.floor(np.exp(u * math.log(hi)))
    return np.clip(c, lo, hi).astype(np.uint32)


def gaussmix_theta_image(width: int, height: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """fp32 [height * width][16]: mixture parameters that vary smoothly over an image
    (row-major pixels), so that neighbouring pixels have nearly equal integrals
    and an estimator's error image shows its spatial structure.  Component c has a
    seeded weight w_c ~ U[0.2,1], width sigma_c ~ U[0.08,0.25], and means
    mu_c = 0.5 + 0.35 sin(2 pi (f_c x / width + p_c)), nu_c = 0.5 + 0.35 sin(2 pi
    (g_c y / height + q_c)) with seeded frequencies f_c, g_c ~ U[0.5,2.5] and phases."""
    r = uniform01(_key(seed, _T_IMAGE), np.arange(24, dtype=np.uint64)).reshape(4, 6)
    w = 0.2 + 0.8 * r[:, 0]
    sg = 0.08 + 0.17 * r[:, 1]
    f, g = 0.5 + 2.0 * r[:, 2], 0.5 + 2.0 * r[:, 3]
    x = (np.arange(width, dtype=np.float64) + 0.5) / width
    y = (np.arange(height, dtype=np.float64) + 0.5) / height
    th = np.empty((height, width, 4, 4), np.float64)
    for c in range(4):
        th[:, :, c, 0] = w[c]
        th[:, :, c, 1] = 0.5 + 0.35 * np.sin(2 * np.pi * (f[c] * x[None, :] + r[c, 4]))
        th[:, :, c, 2] = 0.5 + 0.35 * np.sin(2 * np.pi * (g[c] * y[:, None] + r[c, 5]))
        th[:, :, c, 3] = sg[c]
    return th.reshape(height * width, 16).astype(np.float32)


def scene_theta(width: int, height: int, freq: float = 8.0, occluder: bool = True) -> np.ndarray:
    """fp32 [height * width][16]: per-pixel parameters of the procedural scene
    (row-major pixels): the pixel's footprint on the ground plane (the image
    covers [0, width/height] x [0, 1], square pixels), then the scene shared by
    all pixels -- a square light of side 0.3 and radiance 1 at height 1 above the
    image centre, a sphere of radius 0.12 centred at 35 % of that height, offset
    towards the origin, and a checkerboard of `freq` cells per unit length."""
    aspect = width / height
    p = np.arange(width * height)
    th = np.zeros((width * height, 16), np.float64)
    th[:, 0] = (p % width) / height
    th[:, 1] = (p // width) / height
    th[:, 2] = th[:, 3] = 1.0 / height
    th[:, 4:9] = [0.5 * aspect, 0.5, 1.0, 0.3, 1.0]
    th[:, 9:13] = [0.45 * aspect, 0.45, 0.35, 0.12 if occluder else 0.0]
    th[:, 13] = freq
    return th.astype(np.float32)


def gaussmix_target(theta_star: np.ndarray) -> np.ndarray:
    """Synthetic target image: the exact integral of the mixture at parameters theta_star.

    Used only to build a seeded target for the squared-error loss; the QMC
    path never evaluates it.
    """
    try:
        from scipy.special import erf
    except ImportError:  # pragma: no cover - scipy is present on both machines
        erf = np.vectorize(math.erf)
    th = np.asarray(theta_star, dtype=np.float64).reshape(-1, 4, 4)
    w, mu, nu, sg = th[..., 0], th[..., 1], th[..., 2], th[..., 3]
    r2 = math.sqrt(2.0)

    def g1(m):
        return sg * math.sqrt(math.pi / 2) * (erf((1 - m) / (sg * r2)) + erf(m / (sg * r2)))

    return (w * g1(mu) ** 3 * g1(nu) ** 3).sum(axis=1)
