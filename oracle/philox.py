"""Philox4x32-10 counter-based generator, restated from its published definition
(Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as easy as 1, 2, 3",
SC'11).  Test oracle only.

Each call maps a 128-bit counter and a 64-bit key to four 32-bit words through
ten rounds.  A round multiplies counter words 0 and 2 by the constants
0xD2511F53 and 0xCD9E8D57 (full 64-bit products), and mixes the high halves with
the other two counter words and the key; the key is advanced by the Weyl
constants 0x9E3779B9 / 0xBB67AE85 between rounds.

Stream convention of the MapElites operators: the random words of candidate
``cand`` in iteration ``it`` under seed ``seed`` are the concatenation over
block = 0, 1, 2, ... of philox(counter=(block, cand, it_lo, it_hi),
key=(seed_lo, seed_hi)).
"""
from __future__ import annotations

MASK = 0xFFFFFFFF
M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85


def philox4x32_10(ctr, key):
    c0, c1, c2, c3 = (int(x) & MASK for x in ctr)
    k0, k1 = (int(x) & MASK for x in key)
    for r in range(10):
        if r:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0
        p1 = M1 * c2
        c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0) & MASK, p1 & MASK, ((p0 >> 32) ^ c3 ^ k1) & MASK, p0 & MASK
    return c0, c1, c2, c3


class WordStream:
    """Sequential 32-bit words of one (seed, iteration, candidate) stream."""

    def __init__(self, seed: int, iteration: int, cand: int):
        self.key = (seed & MASK, (seed >> 32) & MASK)
        self.it = (iteration & MASK, (iteration >> 32) & MASK)
        self.cand = cand & MASK
        self.block = 0
        self.buf = []
        self.used = 0

    def next(self) -> int:
        if not self.buf:
            self.buf = list(philox4x32_10((self.block, self.cand, self.it[0], self.it[1]), self.key))
            self.block += 1
        self.used += 1
        return self.buf.pop(0)


def uniform_index(word: int, n: int) -> int:
    """Map a 32-bit word to [0, n) by the high half of word * n."""
    return (int(word) * int(n)) >> 32
