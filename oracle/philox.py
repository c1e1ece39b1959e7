"""Philox4x32-10, restated from its published definition.

Test infrastructure only (see ``oracle/__init__.py``).

Source: J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel Random
Numbers: As Easy as 1, 2, 3", SC'11, Sec. 3.2 (Philox): a 4-word counter
block is passed through R = 10 rounds.  Each round multiplies words 0 and 2
by the constants M0 = 0xD2511F53 and M1 = 0xCD9E8D57 (32x32 -> 64-bit), and
forms the new block from the high/low halves of the two products, XORed
with the untouched words 1 and 3 and with the two round-key words.  The
round key starts at the user key (k0, k1) and is advanced between rounds by
the Weyl constants W0 = 0x9E3779B9, W1 = 0xBB67AE85 (mod 2^32).

Pinned in the tests against the Philox4x32-10 generator of the cuRAND host
library, run (not read) through its public API.
"""

import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
_LO32 = np.uint64(0xFFFFFFFF)
_SHIFT = np.uint64(32)


def philox4x32_10(counter, key):
    """Return the 4 output words for each counter block.

    counter: integer array [..., 4] (values < 2**32), words c0..c3.
    key:     integer array [..., 2] broadcastable to counter[..., :2], words k0, k1.
    Returns a uint32 array [..., 4].
    """
    counter = np.asarray(counter, dtype=np.uint64)
    key = np.asarray(key, dtype=np.uint64)
    c0, c1, c2, c3 = (counter[..., i] for i in range(4))
    k0 = np.broadcast_to(key[..., 0], c0.shape).copy()
    k1 = np.broadcast_to(key[..., 1], c0.shape).copy()
    m0 = np.uint64(M0)
    m1 = np.uint64(M1)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + np.uint64(W0)) & _LO32
            k1 = (k1 + np.uint64(W1)) & _LO32
        prod0 = m0 * c0          # both factors < 2**32: exact in uint64
        prod1 = m1 * c2
        hi0, lo0 = prod0 >> _SHIFT, prod0 & _LO32
        hi1, lo1 = prod1 >> _SHIFT, prod1 & _LO32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def split_seed(seed):
    """64-bit seed -> Philox key words (k0 = low 32 bits, k1 = high 32 bits)."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint64)
