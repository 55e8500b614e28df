"""Philox4x32-10 counter-based generator, written out from its published definition.

TEST INFRASTRUCTURE ONLY: this module belongs to the CPU oracle. Only tests, the smoke check and
the CPU-baseline leg of the benchmark may import it; the CUDA library never does.

Definition (Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3", SC'11):
the state is a 128-bit counter (four 32-bit words) and a 64-bit key (two words).  One round
multiplies words 0 and 2 by two fixed odd constants, keeps both halves of each 64-bit product,
and recombines them with words 1 and 3 and the round key.  The key is advanced by two Weyl
constants between rounds.  Ten rounds give the "-10" variant.

The paper (Alg. 3, Alg. 4) only asks for uniform sampling with replacement and random sign flips;
which generator draws them is left open.  A counter-based generator makes every draw a pure
function of (seed, decomposition, iteration, mode, sample), so the oracle and the GPU can be
written independently and still agree bit for bit.

Pinned against: cuRAND's host-side PHILOX4_32_10 generator (tests/test_oracle_philox.py).
"""
import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint32(0x9E3779B9)
_W1 = np.uint32(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)


def _mulhilo(m, x):
    """Full 64-bit product of a 32-bit constant and 32-bit words, split into (hi, lo)."""
    p = m * x.astype(np.uint64)
    return (p >> np.uint64(32)).astype(np.uint32), (p & _MASK).astype(np.uint32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Apply Philox4x32-10 to counters (c0..c3) under key (k0, k1).

    All arguments broadcast; each is an integer array (or scalar) of 32-bit words.
    Returns a tuple of four uint32 arrays (the output words 0..3).
    """
    x0 = np.asarray(c0, dtype=np.uint32)
    x1 = np.asarray(c1, dtype=np.uint32)
    x2 = np.asarray(c2, dtype=np.uint32)
    x3 = np.asarray(c3, dtype=np.uint32)
    x0, x1, x2, x3 = np.broadcast_arrays(x0, x1, x2, x3)
    key0 = np.asarray(k0, dtype=np.uint32)
    key1 = np.asarray(k1, dtype=np.uint32)
    with np.errstate(over="ignore"):
        for rnd in range(10):
            if rnd > 0:
                key0 = (key0 + _W0).astype(np.uint32)
                key1 = (key1 + _W1).astype(np.uint32)
            hi0, lo0 = _mulhilo(_M0, x0)
            hi1, lo1 = _mulhilo(_M1, x2)
            x0, x1, x2, x3 = (hi1 ^ x1 ^ key0, lo1, hi0 ^ x3 ^ key1, lo0)
    return (np.asarray(x0, dtype=np.uint32), np.asarray(x1, dtype=np.uint32),
            np.asarray(x2, dtype=np.uint32), np.asarray(x3, dtype=np.uint32))


def seed_to_key(seed):
    """64-bit seed -> Philox key words (low word first)."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return np.uint32(seed & 0xFFFFFFFF), np.uint32(seed >> 32)
