"""Philox4x32-10 counter-based generator, vectorised over counters with numpy.

Definition: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11 -- the Philox-4x32 bijection with 10 rounds.  Each round maps
the counter (c0, c1, c2, c3) under key (k0, k1) to

    hi0:lo0 = M0 * c0,   hi1:lo1 = M1 * c2        (32x32 -> 64-bit products)
    (c0, c1, c2, c3) <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)

and bumps the key by the Weyl constants (W0, W1) between rounds.

This module draws only synthetic inputs.  The same bijection is written a
second time in CUDA (synthetic/csrc/synth_gen.cu) so that the device can fill
full-size inputs; the two are compared bit for bit by the tests.
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = 0x9E3779B9
W1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32(c0, c1, c2, c3, k0, k1, rounds=10):
    """Apply Philox4x32 to arrays of 32-bit counter words under one key.

    c0..c3 are integer arrays (broadcastable); k0, k1 are Python ints.
    Returns four uint32 arrays.
    """
    c0 = np.asarray(c0, dtype=np.uint64) & _MASK32
    c1 = np.asarray(c1, dtype=np.uint64) & _MASK32
    c2 = np.asarray(c2, dtype=np.uint64) & _MASK32
    c3 = np.asarray(c3, dtype=np.uint64) & _MASK32
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    key0, key1 = int(k0) & 0xFFFFFFFF, int(k1) & 0xFFFFFFFF
    for r in range(rounds):
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(key0), lo1,
                          hi0 ^ c3 ^ np.uint64(key1), lo0)
        key0 = (key0 + W0) & 0xFFFFFFFF
        key1 = (key1 + W1) & 0xFFFFFFFF
    return (c0.astype(np.uint32), c1.astype(np.uint32),
            c2.astype(np.uint32), c3.astype(np.uint32))
