"""Philox4x32-10 counter-based generator (test infrastructure).

Written from its published definition (Salmon, Moraes, Dror & Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC 2011): a 128-bit counter and a 64-bit key; each of
the 10 rounds multiplies two counter words by M0 = 0xD2511F53 and M1 = 0xCD9E8D57
(full 64-bit products), permutes and XORs the halves with the key, and the key is
bumped by the Weyl constants W0 = 0x9E3779B9, W1 = 0xBB67AE85 between rounds.

The sampler draws all its random numbers from this generator at fixed counters, so the
GPU path (its own implementation of the same definition) and the oracle draw
identical bits. Conversions used by the sampler:

* u53(a, b) = ((a >> 5) 2^26 + (b >> 6)) 2^-53 in [0, 1) -- exact in float64.
* u32(a)    = (a + 1/2) 2^-32 in (0, 1)                    -- exact in float64.
* u24(a)    = (a >> 8) 2^-24 in [0, 1)                      -- exact.
* ranged index: (a * n) >> 32 in [0, n).
"""
M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """Four 32-bit output words for counter (c0..c3) and key (k0, k1)."""
    c0, c1, c2, c3 = [int(x) & MASK for x in ctr]
    k0, k1 = [int(x) & MASK for x in key]
    for r in range(10):
        if r > 0:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> 32, p0 & MASK
        hi1, lo1 = p1 >> 32, p1 & MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & MASK, lo1, (hi0 ^ c3 ^ k1) & MASK, lo0
    return c0, c1, c2, c3


def u53(a, b):
    return ((a >> 5) * 67108864.0 + (b >> 6)) * (1.0 / 9007199254740992.0)


def u32(a):
    return (a + 0.5) * (1.0 / 4294967296.0)


def u24(a):
    return (a >> 8) * (1.0 / 16777216.0)


def ranged(a, n):
    return (a * n) >> 32


class Stream:
    """Sequential words from consecutive counters c0 = base, base + 1, ... with c1..c3 fixed."""

    def __init__(self, key, c0, c1, c2, c3):
        self.key = key
        self.c = [c0, c1, c2, c3]
        self.buf = []

    def word(self):
        if not self.buf:
            self.buf = list(philox4x32_10(self.c, self.key))
            self.c[0] += 1
        return self.buf.pop(0)
