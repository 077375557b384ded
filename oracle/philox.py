"""Counter-based Philox4x32-10 generator and the Gaussian test matrix -- TEST INFRASTRUCTURE ONLY.

The randomized SVD of Sec. 4.3 multiplies X by a random Gaussian matrix; the
paper leaves the generator open.  The CUDA library draws it on the device from
Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11), so the oracle re-implements that published definition here
independently, in plain Python integers, to check the device generator bit for
bit.

Element e of the test matrix (column-major, m x l) uses counter
(e // 4 mod 2^32, e // 4 >> 32, 0x0D3D0001, 0) and key (seed mod 2^32, seed >> 32);
the four 32-bit outputs x0..x3 become two Box-Muller pairs with
u = (x + 0.5) * 2^-32: g0, g1 from (x0, x1) and g2, g3 from (x2, x3),
g_even = sqrt(-2 ln u_a) cos(2 pi u_b), g_odd = sqrt(-2 ln u_a) sin(2 pi u_b).
Element e takes output e mod 4.
"""
from __future__ import annotations

import math

import numpy as np

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK = 0xFFFFFFFF
STREAM_SKETCH = 0x0D3D0001


def philox4x32_10(ctr, key):
    """One Philox4x32 block with 10 rounds; ctr is 4 words, key is 2 words."""
    c0, c1, c2, c3 = (int(v) & MASK for v in ctr)
    k0, k1 = (int(v) & MASK for v in key)
    for rnd in range(10):
        if rnd:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> 32, p0 & MASK
        hi1, lo1 = p1 >> 32, p1 & MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def gaussian_block(block: int, seed: int):
    x = philox4x32_10((block & MASK, block >> 32, STREAM_SKETCH, 0), (seed & MASK, seed >> 32))
    u = [(v + 0.5) * 2.0 ** -32 for v in x]
    ra = math.sqrt(-2.0 * math.log(u[0]))
    rb = math.sqrt(-2.0 * math.log(u[2]))
    return (ra * math.cos(2 * math.pi * u[1]), ra * math.sin(2 * math.pi * u[1]),
            rb * math.cos(2 * math.pi * u[3]), rb * math.sin(2 * math.pi * u[3]))


def sketch_matrix(m: int, l: int, seed: int) -> np.ndarray:
    """The m x l Gaussian test matrix the device draws for a given seed."""
    total = m * l
    flat = np.empty(total)
    for blk in range((total + 3) // 4):
        g = gaussian_block(blk, seed)
        for t in range(4):
            e = 4 * blk + t
            if e < total:
                flat[e] = g[t]
    return flat.reshape(l, m).T.copy()       # column-major element order
