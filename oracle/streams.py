"""Where every random number of the method comes from (oracle side).

TEST INFRASTRUCTURE ONLY (CPU oracle).  The CUDA library implements the same stream layout on its
own; the two share no code.

The paper draws four kinds of random quantities:
  * the S sampled multi-indices of every mode update (§3.2, Alg. 3: uniform, with replacement,
    drawn afresh for every mode of every outer iteration, §4.2);
  * the fixed set of P_hat tensor entries used by the sampled fit (§3.4, fixed for a run, §4.2);
  * the random initial factor matrices (Alg. 3 / Alg. 5, initialization step);
  * the random sign flips D_n of the mixing preprocess (§2.2 FJLT, Alg. 5).

Each is a Philox4x32-10 draw keyed by the 64-bit run seed.  Counter words:
  word 0 : the item index (sample j, fit entry j, factor row i, sign index i)
  word 1 : (stream << 8) | (block << 4) | mode
  word 2 : outer iteration t (samples), factor column group r // 4 (init), else 0
  word 3 : decomposition index b inside a batch (0 for a single run)
with stream 0 = LS samples, 1 = fit entries, 2 = initial factors, 3 = signs.

Integer mapping: index in [0, I) = floor(w * I / 2**32) (a 64-bit multiply-high; the bias is at
most I / 2**32).  Uniform value in [0, 1) = (w >> 8) * 2**-24 (exact in fp32 and fp64).
Sign = +1 when the low bit of the word is 0, else -1.
"""
import numpy as np

from .philox import philox4x32_10, seed_to_key

STREAM_SAMPLES = 0
STREAM_FIT = 1
STREAM_INIT = 2
STREAM_SIGNS = 3


def _word1(stream, block, mode):
    return np.uint32((stream << 8) | (block << 4) | mode)


def _index_from_word(w, extent):
    return ((w.astype(np.uint64) * np.uint64(extent)) >> np.uint64(32)).astype(np.int64)


def ls_sample_indices(seed, b, t, n, S, dims):
    """Sampled multi-indices for the mode-n update of outer iteration t (Alg. 3, §3.2).

    Returns an (S, N) int64 array of 0-based indices; column n is left at 0 (the mode being
    solved for is not sampled).  The k-th mode other than n (in increasing order) takes word
    k % 4 of Philox block k // 4.
    """
    N = len(dims)
    k0, k1 = seed_to_key(seed)
    j = np.arange(S, dtype=np.uint64).astype(np.uint32)
    idx = np.zeros((S, N), dtype=np.int64)
    others = [m for m in range(N) if m != n]
    blocks = {}
    for k, m in enumerate(others):
        blk = k // 4
        if blk not in blocks:
            blocks[blk] = philox4x32_10(j, _word1(STREAM_SAMPLES, blk, n), np.uint32(t),
                                        np.uint32(b), k0, k1)
        idx[:, m] = _index_from_word(blocks[blk][k % 4], dims[m])
    return idx


def fit_sample_indices(seed, b, P_hat, dims):
    """The fixed set of P_hat entries used by the sampled fit (§3.4), i.i.d. uniform.

    Returns a (P_hat, N) int64 array; mode m takes word m % 4 of Philox block m // 4.
    """
    N = len(dims)
    k0, k1 = seed_to_key(seed)
    j = np.arange(P_hat, dtype=np.uint64).astype(np.uint32)
    idx = np.zeros((P_hat, N), dtype=np.int64)
    blocks = {}
    for m in range(N):
        blk = m // 4
        if blk not in blocks:
            blocks[blk] = philox4x32_10(j, _word1(STREAM_FIT, blk, 0), np.uint32(0),
                                        np.uint32(b), k0, k1)
        idx[:, m] = _index_from_word(blocks[blk][m % 4], dims[m])
    return idx


def init_factor(seed, b, n, I, R):
    """Random initial factor for mode n: I x R entries uniform in [0, 1) (Alg. 3 initialization)."""
    k0, k1 = seed_to_key(seed)
    i = np.arange(I, dtype=np.uint64).astype(np.uint32)
    A = np.zeros((I, R), dtype=np.float64)
    for g in range((R + 3) // 4):
        w = philox4x32_10(i, _word1(STREAM_INIT, 0, n), np.uint32(g), np.uint32(b), k0, k1)
        for q in range(4):
            r = 4 * g + q
            if r < R:
                A[:, r] = (w[q] >> np.uint32(8)).astype(np.float64) * 2.0 ** -24
    return A


def sign_vector(seed, b, n, I):
    """Diagonal of the random sign-flip operator D_n (§2.2 FJLT step one, Alg. 5)."""
    k0, k1 = seed_to_key(seed)
    i = np.arange(I, dtype=np.uint64).astype(np.uint32)
    w = philox4x32_10(i, _word1(STREAM_SIGNS, 0, n), np.uint32(0), np.uint32(b), k0, k1)[0]
    return np.where((w & np.uint32(1)) == 0, 1.0, -1.0)
