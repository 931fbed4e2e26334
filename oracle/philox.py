"""Counter-based Gaussian sketch generator (oracle side; test infrastructure only).

Definition 3.1 asks for a TT whose core n holds i.i.d. N(0, 1/(l_{n-1} I_n l_n))
entries. To let the device draw the same sketch from a seed, both sides
implement one published counter-based generator, Philox4x32-10 (Salmon, Moraes,
Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11), and the
Box-Muller transform. This file is the oracle's own NumPy implementation; the
CUDA side has its own.

Entry e (C order) of core n (0-based) of the sketch with seed s:
  pair p = e // 2; counter = (p mod 2^32, p div 2^32, n, 0x7474726e);
  key = (s mod 2^32, s div 2^32); (x0, x1, x2, x3) = Philox4x32-10(counter, key)
  u1 = ((x0 << 20) | (x1 >> 12)) + 1/2) 2^-52, u2 likewise from (x2, x3)
  (both exact in float64, inside (0, 1));
  z0 = sqrt(-2 ln u1) cos(2 pi u2), z1 = sqrt(-2 ln u1) sin(2 pi u2);
  entry = (z0 if e is even else z1) / sqrt(l_{n-1} I_n l_n).
"""
from __future__ import annotations

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)
TAG = 0x7474726E


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on uint32 arrays (computed in uint64).
    One round: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2 (full 64-bit
    products); c := (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key is
    advanced by the Weyl constants (W0, W1) between rounds."""
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) & _MASK for x in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK
    for r in range(10):
        if r > 0:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return c0, c1, c2, c3


def _u52(a, b):
    bits = (a << np.uint64(20)) | (b >> np.uint64(12))
    return (bits.astype(np.float64) + 0.5) * (2.0 ** -52)


def gaussian_sketch_philox(seed, dims, ells):
    """Gaussian TT sketch of Definition 3.1 with ranks ells (length N+1) drawn
    from the counter-based generator described in the module docstring."""
    seed = int(seed)
    k0 = np.uint64(seed & 0xFFFFFFFF)
    k1 = np.uint64((seed >> 32) & 0xFFFFFFFF)
    cores = []
    for n, I in enumerate(dims):
        r0, r1 = int(ells[n]), int(ells[n + 1])
        E = r0 * I * r1
        e = np.arange(E, dtype=np.uint64)
        p = e >> np.uint64(1)
        x0, x1, x2, x3 = philox4x32_10(p & _MASK, p >> np.uint64(32),
                                       np.full(E, n, dtype=np.uint64), np.full(E, TAG, dtype=np.uint64),
                                       k0, k1)
        u1 = _u52(x0, x1)
        u2 = _u52(x2, x3)
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.where((e & np.uint64(1)) == 0, r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2))
        cores.append((z / np.sqrt(r0 * I * r1)).reshape(r0, I, r1))
    return cores
