"""Seeded synthetic inputs shared by the GPU path, its tests and the benchmark.

This module generates *inputs only*: quark propagators S^{ab}_{alpha beta}(t, x)
with the layout the paper reads them in (one time slice at a time, sink colour
and spin first, then source colour and spin; Sec. IV and App. A) and random
SU(3) matrices for gauge-covariance checks.  It holds none of the correlator
arithmetic (blocks, Wick sums, term reduction) and imports nothing else from
the package, so the independent CPU reference and the CUDA path can both be
fed from it without sharing any of the method.

Random numbers come from a counter-based SplitMix64 (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): the value for
counter i of a stream with key k is mix64(k + (i + 1) * GOLDEN_GAMMA).  Complex
Gaussians use the Box-Muller transform with variance 1/2 per component, so that
E|S|^2 = 1 per entry.

Propagator layout (row-major):  S[src][t][x][a][alpha][b][beta], complex,
x = (z * L + y) * L + x_ (lexicographic), a, b in 0..2, alpha, beta in 0..3.
"""
from __future__ import annotations

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

#: seed of the deuteron workload (u propagator; d uses seed + 1)
SEED_DEUTERON = 0x24110001


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied elementwise to uint64 values."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, *tags: int) -> np.uint64:
    """Derive a stream key from a seed and integer tags (flavour, source, ...)."""
    k = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        for tag in tags:
            k = mix64(k + GOLDEN_GAMMA * np.uint64(tag + 1))
    return np.uint64(k)


def splitmix_block(key: np.uint64, start: int, count: int) -> np.ndarray:
    """Counter values start .. start+count-1 of the stream `key` (uint64)."""
    i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(key + i * GOLDEN_GAMMA)


def gaussian_complex(key: np.uint64, start: int, count: int) -> np.ndarray:
    """`count` i.i.d. complex Gaussians (variance 1/2 per component), complex128."""
    r = splitmix_block(key, 2 * start, 2 * count)
    u1 = ((r[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)
    u2 = (r[1::2] >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    rad = np.sqrt(-np.log(u1))
    ang = 2.0 * np.pi * u2
    return rad * np.cos(ang) + 1j * (rad * np.sin(ang))


def propagator(seed: int, flavour: int, L: int, T: int, n_src: int,
               dtype=np.complex128, t_range=None) -> np.ndarray:
    """Synthetic propagator S_f[src][t][x][3][4][3][4] (i.i.d. complex Gaussian).

    flavour: 0 = u, 1 = d.  Every (flavour, src) pair is its own stream; entry n
    of that stream is the n-th complex number of the flat [t][x][a][al][b][be]
    index, so any sub-range of time slices can be regenerated on its own.
    `t_range` = (t0, t1) returns only slices t0..t1-1 (shape [n_src][t1-t0]...).
    """
    V = L * L * L
    per_t = V * 144
    t0, t1 = (0, T) if t_range is None else t_range
    out = np.empty((n_src, t1 - t0, V, 3, 4, 3, 4), dtype=dtype)
    for s in range(n_src):
        key = stream_key(seed, flavour, s)
        vals = gaussian_complex(key, t0 * per_t, (t1 - t0) * per_t)
        out[s] = vals.reshape(t1 - t0, V, 3, 4, 3, 4).astype(dtype)
    return out


def random_su3(rng: np.random.Generator, n: int) -> np.ndarray:
    """n Haar-ish random SU(3) matrices (QR of complex Gaussians, det fixed to 1)."""
    z = (rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=1, axis2=2)
    q = q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(q)
    q = q / (det ** (1.0 / 3.0))[:, None, None]
    return q


#: The synthetic workloads: lattice extent L, time extent T, sources, storage.
WORKLOADS = {
    "deuteron": dict(L=4, T=8, n_src=1, dtype="c128", seed=SEED_DEUTERON),
    "he3": dict(L=8, T=16, n_src=2, dtype="c128", seed=0x24110003),
    "he4": dict(L=16, T=32, n_src=4, dtype="c64", seed=0x24110004),
    "li7": dict(L=24, T=48, n_src=1, dtype="c64", seed=0x24110007),
    "batched": dict(L=32, T=64, n_src=2, dtype="c64", seed=0x24110005, n_cfg=64),
}
