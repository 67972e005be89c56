"""Counter-based Gaussian test matrices for the randomized HSS construction.

Test infrastructure only: nothing on the product path imports this module.

The black-box construction (Section 3.1, 3.2) draws an independent i.i.d.
Gaussian test matrix Omega^[l] at every level.  Its size depends on ranks
found at finer levels, so the matrices cannot be generated ahead of time and
passed in.  Both the oracle and the CUDA library therefore evaluate the same
counter-based generator, each from its published definition:

* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
  as 1, 2, 3", SC 2011): 10 rounds of two 32x32->64 multiplies with the
  constants M0 = 0xD2511F53, M1 = 0xCD9E8D57 and Weyl key increments
  W0 = 0x9E3779B9, W1 = 0xBB67AE85.
* Box-Muller (Box and Muller, 1958) on the first two output words.

Entry (row, col) of the level-l, attempt-a test matrix uses counter
(row, col, l, a) and key (seed mod 2^32, seed div 2^32); its real and imaginary
parts are independent standard normals.
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint32(0x9E3779B9)
W1 = np.uint32(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)


def _mulhilo(a, b):
    p = a.astype(np.uint64) * b
    return (p >> np.uint64(32)).astype(np.uint32), (p & MASK32).astype(np.uint32)


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds.

    ctr: uint32 array (..., 4); key: uint32 array (..., 2) (broadcastable).
    Returns uint32 array (..., 4).
    """
    c = [np.asarray(ctr[..., i], dtype=np.uint32) for i in range(4)]
    k0 = np.asarray(key[..., 0], dtype=np.uint32).copy()
    k1 = np.asarray(key[..., 1], dtype=np.uint32).copy()
    with np.errstate(over="ignore"):
        for rnd in range(10):
            if rnd > 0:
                k0 = (k0 + W0).astype(np.uint32)
                k1 = (k1 + W1).astype(np.uint32)
            hi0, lo0 = _mulhilo(c[0], M0)
            hi1, lo1 = _mulhilo(c[2], M1)
            c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return np.stack(c, axis=-1)


def gaussian_matrix(seed, level, attempt, rows, cols):
    """Complex test matrix Omega (rows x cols), complex128.

    Re and Im of every entry are independent N(0, 1) (Section 3.1: i.i.d.
    Gaussian entries).
    """
    if rows == 0 or cols == 0:
        return np.zeros((rows, cols), dtype=np.complex128)
    i = np.arange(rows, dtype=np.uint32)[:, None]
    j = np.arange(cols, dtype=np.uint32)[None, :]
    ctr = np.empty((rows, cols, 4), dtype=np.uint32)
    ctr[..., 0] = i
    ctr[..., 1] = j
    ctr[..., 2] = np.uint32(level)
    ctr[..., 3] = np.uint32(attempt)
    seed = int(seed)
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)
    x = philox4x32_10(ctr, key)
    u1 = (x[..., 0].astype(np.float64) + 0.5) * 2.0 ** -32
    u2 = (x[..., 1].astype(np.float64) + 0.5) * 2.0 ** -32
    rad = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    return rad * np.cos(ang) + 1j * (rad * np.sin(ang))
