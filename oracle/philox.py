"""Philox4x32-10 counter-based generator and Box–Muller normals (test infrastructure only).

Philox4x32-10 is written from its published definition (Salmon, Moraes, Dror & Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC'11): a 128-bit counter (x0, x1, x2, x3) and a 64-bit key (k0, k1);
ten rounds, each

    (hi0, lo0) = M0 * x0,  (hi1, lo1) = M1 * x2      (64-bit products of 32-bit words)
    (x0, x1, x2, x3) <- (hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0)

with the key bumped by the Weyl constants (W0, W1) between rounds.

The paper draws its G(0,1) variates with a Box–Muller transform (§3.2); the mapping from counters to
variates used here (stream layout, uniform spacing) is this code base's reading, identical on the GPU:

* key = (seed mod 2^32, seed div 2^32); counter = (group, step, chain, stream);
* each 32-bit word x becomes u = (2*floor(x / 2^9) + 1) * 2^-24, an odd multiple of 2^-24 in (0, 1)
  that is exact in float32 and float64;
* (z0, z1) = sqrt(-2 ln u0) * (cos 2 pi u1, sin 2 pi u1), (z2, z3) likewise from (u2, u3).
"""
from __future__ import annotations

import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK32 = 0xFFFFFFFF

STREAM_T = 0   # pixel-space messenger draw (Alg. 1, t-update)
STREAM_S = 1   # Fourier-space signal draw (Alg. 1, s-update)
STREAM_PROBE = 5  # Rademacher probes for stochastic traces
STREAM_BAND = 6   # chi-square variates of the band-power draw (hierarchical sampler)
STREAM_T2 = 8     # spin-2: messenger draw of the second shear component
STREAM_SB = 9     # spin-2: Fourier-space draw of the B mode


def philox4x32_10(ctr: np.ndarray, key: tuple[int, int]) -> np.ndarray:
    """Apply Philox4x32-10 to counters ``ctr`` (uint array [..., 4]) under ``key`` -> uint32 [..., 4]."""
    x = np.asarray(ctr, dtype=np.uint64) & np.uint64(MASK32)
    x0, x1, x2, x3 = (x[..., i].copy() for i in range(4))
    k0 = int(key[0]) & MASK32
    k1 = int(key[1]) & MASK32
    m0 = np.uint64(M0)
    m1 = np.uint64(M1)
    mask = np.uint64(MASK32)
    sh = np.uint64(32)
    for r in range(10):
        p0 = m0 * x0
        p1 = m1 * x2
        hi0, lo0 = p0 >> sh, p0 & mask
        hi1, lo1 = p1 >> sh, p1 & mask
        x0, x1, x2, x3 = (hi1 ^ x1 ^ np.uint64(k0), lo1, hi0 ^ x3 ^ np.uint64(k1), lo0)
        k0 = (k0 + W0) & MASK32
        k1 = (k1 + W1) & MASK32
    return np.stack([x0, x1, x2, x3], axis=-1).astype(np.uint32)


def seed_key(seed: int) -> tuple[int, int]:
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return (seed & MASK32, seed >> 32)


def to_uniform(x: np.ndarray) -> np.ndarray:
    """32-bit word -> odd multiple of 2^-24 in (0, 1) (exact in float32 and float64)."""
    top = (np.asarray(x, dtype=np.uint64) >> np.uint64(9)).astype(np.float64)
    return (2.0 * top + 1.0) * 2.0 ** -24


def box_muller(u0: np.ndarray, u1: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Two independent N(0,1) variates from two uniforms (Box & Muller 1958)."""
    r = np.sqrt(-2.0 * np.log(u0))
    a = 2.0 * np.pi * u1
    return r * np.cos(a), r * np.sin(a)


def normals4(groups: np.ndarray, step: int, chain: int, stream: int, seed: int) -> np.ndarray:
    """Four N(0,1) variates per counter group -> float64 [len(groups), 4]."""
    g = np.asarray(groups, dtype=np.uint64)
    ctr = np.stack([g,
                    np.full_like(g, np.uint64(int(step) & MASK32)),
                    np.full_like(g, np.uint64(int(chain) & MASK32)),
                    np.full_like(g, np.uint64(int(stream) & MASK32))], axis=-1)
    x = philox4x32_10(ctr, seed_key(seed))
    u = to_uniform(x)
    z0, z1 = box_muller(u[:, 0], u[:, 1])
    z2, z3 = box_muller(u[:, 2], u[:, 3])
    return np.stack([z0, z1, z2, z3], axis=-1)
