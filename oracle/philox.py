"""Oracle: Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC 2011), used to draw the
training batch of each step (uniform random blocks).

TEST INFRASTRUCTURE ONLY.

One round maps counter (c0, c1, c2, c3) and key (k0, k1) to
  (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0)),
with M0 = 0xD2511F53, M1 = 0xCD9E8D57; the key advances by the Weyl constants
(0x9E3779B9, 0xBB67AE85) between rounds; ten rounds.

Batch sampling: for step t and sample i, word (i mod 4) of
philox(counter=(i div 4, t, 0, 0), key=(seed mod 2^32, seed div 2^32)) gives
block = (word * n_blocks) >> 32.
"""
import numpy as np

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK = 0xFFFFFFFF


def philox4x32(ctr, key, rounds=10):
    """ctr: uint64 array [..., 4] holding 32-bit words; key: [..., 2]. Returns uint64 [..., 4]."""
    c = [np.asarray(ctr[..., i], np.uint64) & MASK for i in range(4)]
    k0 = np.asarray(key[..., 0], np.uint64) & MASK
    k1 = np.asarray(key[..., 1], np.uint64) & MASK
    for r in range(rounds):
        p0 = np.uint64(M0) * c[0]
        p1 = np.uint64(M1) * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & np.uint64(MASK)
        hi1, lo1 = p1 >> np.uint64(32), p1 & np.uint64(MASK)
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
        if r + 1 < rounds:
            k0 = (k0 + np.uint64(W0)) & np.uint64(MASK)
            k1 = (k1 + np.uint64(W1)) & np.uint64(MASK)
    return np.stack(c, axis=-1)


def sample_blocks(seed, step, n_samples, n_blocks):
    i = np.arange(n_samples, dtype=np.uint64)
    ctr = np.stack([i // np.uint64(4), np.full_like(i, step), np.zeros_like(i), np.zeros_like(i)], axis=-1)
    key = np.stack([np.full_like(i, seed & MASK), np.full_like(i, (seed >> 32) & MASK)], axis=-1)
    words = philox4x32(ctr, key)
    w = np.take_along_axis(words, (i % np.uint64(4)).astype(np.int64)[:, None], axis=1)[:, 0]
    return ((w * np.uint64(n_blocks)) >> np.uint64(32)).astype(np.int64)
