"""Plain CPU oracle for the QMC hot path (ctypes over ``liboracle.so``).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
cpu_baseline / reference leg of ``bench.py`` may import this package; the
product package never does.  The arithmetic lives in ``qmc_oracle.c`` (plain
C, fp64 integrands, one bit / digit / sample at a time); this module only
marshals numpy arrays and, for speed of the test suite, runs independent
integrals or row ranges on several host threads (ctypes releases the GIL).

Parity unpinned: the exact output bits of ``nested_scramble`` (the paper
names Owen scrambling but prints no algorithm; see ``qmc_oracle.c``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qmc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

SOURCE_SOBOL, SOURCE_LATTICE, SOURCE_PIXEL_LATTICE, SOURCE_RANDOM_LATTICE = 0, 1, 2, 3
RLAT_HASH, RLAT_LFSR = 0, 1
SCRAMBLE_NONE, SCRAMBLE_XOR, SCRAMBLE_NESTED, SCRAMBLE_NESTED_XOR = 0, 1, 2, 3
F_BILINEAR2D, F_GENZ_PRODUCT_PEAK, F_GENZ_OSCILLATORY, F_GAUSSMIX4_6D, F_SCENE4D = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile qmc_oracle.c with gcc (no FMA contraction, so x86 and Arm agree)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        u32, u64, i32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
        P = ctypes.c_void_p
        dbl = ctypes.c_double
        sig = {
            "qo_map_u32_to_unifloat": (ctypes.c_float, [u32]),
            "qo_map_array": (None, [P, u64, P]),
            "qo_bit_reverse": (u32, [u32]),
            "qo_radical_inverse_u32": (u32, [u32, u64]),
            "qo_primitive_polynomials": (u32, [u32, P, u32]),
            "qo_sobol_matrices": (i32, [u32, P, P]),
            "qo_sobol_matrices_wide": (i32, [u32, u32, P, P]),
            "qo_sobol_u64": (u32, [P, u32, u64]),
            "qo_sobol_points_wide": (None, [P, u32, u32, u64, u64, u32, P, P, P]),
            "qo_partition_index": (u64, [u32, u32, u64, u64]),
            "qo_sobol_points_partitioned": (None, [P, u32, u32, u32, u64, u64, u64, u32, P, P, P]),
            "qo_halton_u64": (u32, [u64, u32, u32, u32]),
            "qo_splitmix64": (u64, [u64, u64]),
            "qo_rlat_hash": (u32, [u32, u32, u32, u32, u32]),
            "qo_lfsr_step": (u32, [u32]),
            "qo_rlat_generator": (u32, [u32, u32, u32, u32, u32, u32]),
            "qo_random_lattice_u32": (u32, [u32, u32, u32, u32, u32, u32, u32]),
            "qo_random_lattice_points": (None, [u32, u32, u32, u32, u32, u64, u64, u32, P]),
            "qo_halton_points_partitioned": (None, [u32, u32, P, u32, u64, u64, u64, P]),
            "qo_sobol_u32": (u32, [P, u32]),
            "qo_nested_scramble": (u32, [u32, u32]),
            "qo_sobol_points": (None, [P, u32, u64, u64, u32, P, P, P]),
            "qo_lattice_u32": (u32, [u32, u32, u32, u32]),
            "qo_lattice_points": (None, [P, P, u32, u64, u64, u32, P, P]),
            "qo_hilbert_index": (u32, [u32, u32, u32]),
            "qo_prime": (u32, [u32]),
            "qo_faure": (u32, [u32, u32]),
            "qo_halton_u32": (u32, [u32, u32, u32, u32]),
            "qo_pixel_shift": (u32, [u32, u32, u32]),
            "qo_pixel_lattice_u32": (u32, [u32, u32, u32]),
            "qo_integrate_one": (i32, [u32, u32, u32, u32, P, P, P, u32, P, P, P, P, P, P]),
            "qo_integrate_range": (i32, [u32, u32, u32, u32, P, P, P, u64, P, P, u64, u64, u64, P, P, P, P, P]),
            "qo_integrand": (dbl, [u32, u32, P, P, P]),
            "qo_integrate_partitioned": (i32, [u32, u32, u32, P, u32, u32, u64, P, u32, P, P, P, P, P, P]),
            "qo_gaussmix_f64": (dbl, [P, P]),
            "qo_exact_genz_product_peak": (dbl, [u32, P]),
            "qo_exact_genz_oscillatory": (dbl, [u32, P]),
            "qo_exact_gaussmix": (dbl, [P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _threads(threads):
    return threads or (os.cpu_count() or 1)


def map_u32_to_unifloat(u, threads=None) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.uint32)
    out = np.empty(u.shape, np.float32)
    uf, of = u.reshape(-1), out.reshape(-1)

    def run(r0, n):
        n = min(n, uf.size - r0)
        lib().qo_map_array(uf[r0:].ctypes.data, n, of[r0:].ctypes.data)

    if uf.size:
        _chunked(uf.size, threads if uf.size > (1 << 20) else 1, run)
    return out


def bit_reverse(v: int) -> int:
    return lib().qo_bit_reverse(v)


def radical_inverse_u32(b: int, i: int) -> int:
    return lib().qo_radical_inverse_u32(b, i)


def primitive_polynomials(max_degree: int = 7) -> list[int]:
    buf = np.zeros(4096, np.uint32)
    n = lib().qo_primitive_polynomials(max_degree, _p(buf), buf.size)
    return [int(v) for v in buf[:n]]


def sobol_matrices(s: int, raw_init: np.ndarray) -> np.ndarray:
    raw = np.ascontiguousarray(raw_init, dtype=np.uint32).reshape(-1)
    if raw.size < 7 * s:
        raise ValueError("raw_init needs 7 words per dimension")
    C = np.zeros((s, 32), np.uint32)
    if lib().qo_sobol_matrices(s, _p(raw), _p(C)) != 0:
        raise ValueError("too many dimensions for polynomials of degree <= 7")
    return C


def sobol_matrices_wide(s: int, m: int, raw_init: np.ndarray) -> np.ndarray:
    """u32 [s][m]: generator columns for indices of up to m bits (32 <= m <= 64)."""
    raw = np.ascontiguousarray(raw_init, dtype=np.uint32).reshape(-1)
    if raw.size < 7 * s:
        raise ValueError("raw_init needs 7 words per dimension")
    C = np.zeros((s, m), np.uint32)
    if lib().qo_sobol_matrices_wide(s, m, _p(raw), _p(C)) != 0:
        raise ValueError("bad dimension count or column count")
    return C


def partition_index(b: int, q: int, p: int, J: int) -> int:
    """Global index of the J-th point of processing element p of P = b^q."""
    return lib().qo_partition_index(b, q, p, J)


def nested_scramble(y: int, seed: int) -> int:
    return lib().qo_nested_scramble(y, seed)


def _chunked(count, threads, fn):
    threads = _threads(threads)
    step = max(1, -(-count // threads))
    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(fn, range(0, count, step), [step] * len(range(0, count, step))))


def sobol_points(C, begin, count, mode=SCRAMBLE_NONE, seeds=None, threads=None):
    """(u32 [count][s], f32 [count][s]) of points begin .. begin+count-1."""
    C = np.ascontiguousarray(C, dtype=np.uint32)
    s = C.shape[0]
    seeds = None if seeds is None else np.ascontiguousarray(seeds, dtype=np.uint32)
    u = np.empty((count, s), np.uint32)
    f = np.empty((count, s), np.float32)

    def run(r0, n):
        n = min(n, count - r0)
        lib().qo_sobol_points(_p(C), s, begin + r0, n, mode, _p(seeds),
                              u[r0:].ctypes.data, f[r0:].ctypes.data)

    _chunked(count, threads, run)
    return u, f


def sobol_points_wide(C, begin, count, mode=SCRAMBLE_NONE, seeds=None, threads=None):
    """(u32, f32) [count][s] of points begin .. begin+count-1 (64-bit indices) of the
    wide matrices C [s][m]."""
    C = np.ascontiguousarray(C, dtype=np.uint32)
    s, m = C.shape
    seeds = None if seeds is None else np.ascontiguousarray(seeds, dtype=np.uint32)
    u = np.empty((count, s), np.uint32)
    f = np.empty((count, s), np.float32)

    def run(r0, n):
        n = min(n, count - r0)
        lib().qo_sobol_points_wide(_p(C), m, s, begin + r0, n, mode, _p(seeds),
                                   u[r0:].ctypes.data, f[r0:].ctypes.data)

    if count:
        _chunked(count, threads, run)
    return u, f


def sobol_points_partitioned(C, q, p, j_begin, count, mode=SCRAMBLE_NONE, seeds=None, threads=None):
    """(u32, f32) [count][s]: dimensions 1..s of the points of processing element p
    of 2^q (partitioned by dimension 0 of C [s+1][m]), local indices j_begin.."""
    C = np.ascontiguousarray(C, dtype=np.uint32)
    s, m = C.shape[0] - 1, C.shape[1]
    seeds = None if seeds is None else np.ascontiguousarray(seeds, dtype=np.uint32)
    u = np.empty((count, s), np.uint32)
    f = np.empty((count, s), np.float32)

    def run(r0, n):
        n = min(n, count - r0)
        lib().qo_sobol_points_partitioned(_p(C), m, s, q, p, j_begin + r0, n, mode, _p(seeds),
                                          u[r0:].ctypes.data, f[r0:].ctypes.data)

    if count:
        _chunked(count, threads, run)
    return u, f


def lattice_points(g, shift, begin, count, backward=False, threads=None):
    g = np.ascontiguousarray(g, dtype=np.uint32)
    s = g.shape[0]
    shift = None if shift is None else np.ascontiguousarray(shift, dtype=np.uint32)
    u = np.empty((count, s), np.uint32)
    f = np.empty((count, s), np.float32)

    def run(r0, n):
        n = min(n, count - r0)
        lib().qo_lattice_points(_p(g), _p(shift), s, begin + r0, n, int(backward),
                                u[r0:].ctypes.data, f[r0:].ctypes.data)

    _chunked(count, threads, run)
    return u, f


def random_lattice_points(kind, seed, R, s, width, n_pixels, spp, pixel_begin=0, threads=None):
    """u32 [n_pixels * spp][s]: per-pixel random lattice samples (Alg. 4), R
    superimposed instances."""
    out = np.empty((n_pixels * spp, s), np.uint32)

    def run(q0, n):
        n = min(n, n_pixels - q0)
        lib().qo_random_lattice_points(kind, seed, R, s, width, pixel_begin + q0, n, spp,
                                       out[q0 * spp:].ctypes.data)

    if n_pixels:
        _chunked(n_pixels, threads, run)
    return out


def random_lattice_seeds(seed, width, n, pixel_begin=0):
    """[n][3] per-integral (seed, px, py) rows for integrate(SOURCE_RANDOM_LATTICE)."""
    p = np.arange(pixel_begin, pixel_begin + n, dtype=np.uint64)
    return np.stack([np.full(n, seed, np.uint64), p % width, p // width], axis=1).astype(np.uint32)


def integrate(source, integrand, s, counts, theta, *, C=None, g=None, scramble=0, seeds=None,
              with_grad=False, threads=None):
    """Per-integral QMC estimates (fp64).

    counts [n]; theta [n][P] (fp32); seeds None, [s] shared or [n][s].
    Returns dict(est [n], mass [n], grad [n][16], grad_mass [n][16], grad_scale [n][16]):
    grad the mean of df/dtheta, grad_mass the mean of |df/dtheta|, grad_scale the mean of
    the sum of the absolute values of the terms of each df/dtheta (>= grad_mass)."""
    counts = np.ascontiguousarray(counts, dtype=np.uint32).reshape(-1)
    n = counts.size
    theta = np.ascontiguousarray(theta, dtype=np.float32).reshape(n, -1)
    C = None if C is None else np.ascontiguousarray(C, dtype=np.uint32)
    g = None if g is None else np.ascontiguousarray(g, dtype=np.uint32)
    if seeds is not None:
        seeds = np.asarray(seeds, dtype=np.uint32)
        if seeds.ndim == 1:  # one seed vector shared by every integral
            seeds = np.tile(seeds.reshape(1, s), (n, 1))
        seeds = np.ascontiguousarray(seeds.reshape(n, -1))  # [n][s], or [n][1] pixel shifts
    est = np.zeros(n)
    mass = np.zeros(n)
    grad = np.zeros((n, 16)) if with_grad else None
    gmass = np.zeros((n, 16)) if with_grad else None
    gscale = np.zeros((n, 16)) if with_grad else None

    def run(rng):
        p0, p1 = rng
        rc = lib().qo_integrate_range(
            source, integrand, s, scramble, _p(C), _p(g), _p(seeds), 0 if seeds is None else seeds.shape[1],
            counts.ctypes.data, theta.ctypes.data, theta.shape[1], p0, p1, est.ctypes.data, mass.ctypes.data,
            _p(grad), _p(gmass), _p(gscale))
        if rc != 0:
            raise ValueError("oracle rejected the problem")

    # contiguous ranges of about equal work (samples plus a per-integral overhead), many per
    # thread so the pool stays busy; each integral is still computed alone, in index order
    T = _threads(threads)
    if n:
        cost = np.cumsum(counts.astype(np.float64) + 64.0)
        cuts = np.searchsorted(cost, np.linspace(0.0, cost[-1], min(n, 32 * T) + 1)[1:-1], side="right")
        bounds = sorted({0, n, *[int(c) for c in cuts if 0 < c < n]})
        with ThreadPoolExecutor(T) as ex:
            list(ex.map(run, zip(bounds[:-1], bounds[1:])))
    return {"est": est, "mass": mass, "grad": grad, "grad_mass": gmass, "grad_scale": gscale}


def integrate_partitioned(integrand, s, counts, theta, C, q, elements, *, scramble=0, seeds=None,
                          with_grad=False, threads=None):
    """Estimates of element elements[k] of the Sobol' sequence partitioned across
    2^q elements by dimension 0 of the wide matrices C [s+1][m] (Sec. 2.5.1),
    with counts[k] samples each.  theta [n][P]; seeds None, [s] or [n][s]."""
    counts = np.ascontiguousarray(counts, dtype=np.uint32).reshape(-1)
    n = counts.size
    theta = np.ascontiguousarray(theta, dtype=np.float32).reshape(n, -1)
    C = np.ascontiguousarray(C, dtype=np.uint32)
    m = C.shape[1]
    elements = np.asarray(elements, dtype=np.uint64).reshape(-1)
    if seeds is not None:
        seeds = np.asarray(seeds, dtype=np.uint32)
        if seeds.ndim == 1:
            seeds = np.tile(seeds.reshape(1, s), (n, 1))
        seeds = np.ascontiguousarray(seeds.reshape(n, -1))
    est, mass = np.zeros(n), np.zeros(n)
    grad = np.zeros((n, 16)) if with_grad else None
    gmass = np.zeros((n, 16)) if with_grad else None
    gscale = np.zeros((n, 16)) if with_grad else None

    def one(k):
        rc = lib().qo_integrate_partitioned(
            integrand, s, scramble, _p(C), m, q, int(elements[k]),
            None if seeds is None else seeds[k].ctypes.data, int(counts[k]), theta[k].ctypes.data,
            est[k:].ctypes.data, mass[k:].ctypes.data,
            None if grad is None else grad[k].ctypes.data, None if gmass is None else gmass[k].ctypes.data,
            None if gscale is None else gscale[k].ctypes.data)
        if rc != 0:
            raise ValueError("oracle rejected the problem")

    order = np.argsort(-counts.astype(np.int64), kind="stable")
    with ThreadPoolExecutor(_threads(threads)) as ex:
        list(ex.map(one, order.tolist()))
    return {"est": est, "mass": mass, "grad": grad, "grad_mass": gmass, "grad_scale": gscale}


def integrand(kind, x, theta, s=None):
    x = np.ascontiguousarray(x, dtype=np.float64)
    theta = np.ascontiguousarray(theta, dtype=np.float32)
    grad = np.zeros(16)
    v = lib().qo_integrand(kind, s or x.size, _p(x), _p(theta), _p(grad))
    return v, grad


def gaussmix_f64(x, th) -> float:
    x = np.ascontiguousarray(x, dtype=np.float64)
    th = np.ascontiguousarray(th, dtype=np.float64)
    return lib().qo_gaussmix_f64(_p(x), _p(th))


def exact_genz_product_peak(theta, s) -> float:
    theta = np.ascontiguousarray(theta, dtype=np.float32)
    return lib().qo_exact_genz_product_peak(s, _p(theta))


def exact_genz_oscillatory(theta, s) -> float:
    theta = np.ascontiguousarray(theta, dtype=np.float32)
    return lib().qo_exact_genz_oscillatory(s, _p(theta))


def exact_gaussmix(theta, with_grad=False):
    th = np.ascontiguousarray(theta, dtype=np.float64)
    grad = np.zeros(16)
    v = lib().qo_exact_gaussmix(_p(th), _p(grad) if with_grad else None)
    return (v, grad) if with_grad else v


def hilbert_index(x: int, y: int, k: int) -> int:
    return lib().qo_hilbert_index(x, y, k)


def pixel_shift(px: int, py: int, k: int) -> int:
    return lib().qo_pixel_shift(px, py, k)


def grid_log2(width: int, height: int) -> int:
    """Order k of the smallest 2^k x 2^k grid that covers the image."""
    k = 0
    while (1 << k) < max(width, height):
        k += 1
    return k


def pixel_lattice_points(g, width, n_pixels, spp, pixel_begin=0, height=None):
    """u32 [n_pixels * spp][s]: samples 0..spp-1 of pixels pixel_begin.. (row-major image)."""
    g = np.ascontiguousarray(g, dtype=np.uint32)
    height = height or -(-(pixel_begin + n_pixels) // width)
    k = grid_log2(width, height)
    out = np.empty((n_pixels * spp, g.size), np.uint32)
    for q in range(n_pixels):
        p = pixel_begin + q
        sh = pixel_shift(p % width, p // width, k)
        for i in range(spp):
            for j in range(g.size):
                out[q * spp + i, j] = lib().qo_pixel_lattice_u32(i, int(g[j]), sh)
    return out


def pixel_shifts(width, n, height=None):
    """Per-integral shift words of an image of n pixels (row-major), for integrate(source=2)."""
    height = height or -(-n // width)
    k = grid_log2(width, height)
    return np.array([[pixel_shift(p % width, p // width, k)] for p in range(n)], np.uint32)


HALTON_NONE, HALTON_FAURE, HALTON_LINEAR = 0, 1, 2


def halton_points(s, begin, count, mode=HALTON_NONE, multipliers=None, threads=None):
    """u32 [count][s]: Halton points begin.. (bases = the first s primes)."""
    mult = np.zeros(s, np.uint32) if multipliers is None else np.asarray(multipliers, np.uint32)
    out = np.empty((count, s), np.uint32)

    def run(r0, n):
        for r in range(r0, min(count, r0 + n)):
            for j in range(s):
                out[r, j] = lib().qo_halton_u32((begin + r) & 0xFFFFFFFF, j, mode, int(mult[j]))

    _chunked(count, threads, run)
    return out


def halton_points_partitioned(s, q, p, j_begin, count, mode=HALTON_NONE, multipliers=None, threads=None):
    """u32 [count][s]: dimensions 1..s (bases 3, 5, ..) of the Halton points of
    processing element p of 2^q (partitioned by dimension 0, base 2)."""
    mult = None if multipliers is None else np.ascontiguousarray(multipliers, np.uint32)
    out = np.empty((count, s), np.uint32)

    def run(r0, n):
        n = min(n, count - r0)
        lib().qo_halton_points_partitioned(s, mode, _p(mult), q, p, j_begin + r0, n,
                                           out[r0:].ctypes.data)

    if count:
        _chunked(count, threads, run)
    return out
