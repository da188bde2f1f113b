"""Host Philox4x32-10 and the random test matrices Omega (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Philox4x32-10 is written from its published definition (Salmon, Moraes, Dror,
Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11, Sec. 4.2): a
10-round Feistel-like bijection on four 32-bit words with two 32x32->64
multiplications per round and a Weyl-sequence key schedule.

Omega follows Sec. I-A of the paper: either i.i.d. N(0, 1) entries, or the
"very sparse" entries in {-1, 0, +1} with probabilities {1/2p, 1 - 1/p, 1/2p}.
The paper fixes neither the generator nor the entry-to-stream mapping; this
build's reading (shared by the GPU library, implemented independently there):

* entry (i, j) of the n x k matrix uses counter (i, j // 4, tag, 0) and key
  (seed mod 2^32, seed // 2^32); word j % 4 of the output feeds column j;
* tag 0 = Gaussian, tag 1 = very sparse;
* Gaussian: Box-Muller on word pairs (w0, w1) -> columns 4b (cos), 4b+1 (sin)
  and (w2, w3) -> 4b+2 (cos), 4b+3 (sin), with u = (w + 1/2) 2^-32, computed
  in FP64 and rounded to nearest-even FP32;
* very sparse: T = floor(2^32 / (2p)); w < T -> -1, T <= w < 2T -> +1, else 0.
"""
from __future__ import annotations

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)

TAG_GAUSSIAN = 0
TAG_SPARSE = 1


def _mulhilo(m: np.uint64, x: np.ndarray):
    prod = m * x.astype(np.uint64)
    return (prod >> np.uint64(32)) & _MASK, prod & _MASK


def philox4x32_10(c0, c1, c2, c3, k0: int, k1: int):
    """Philox4x32 with 10 rounds (Salmon et al. SC'11, Sec. 4.2).

    Counters are broadcastable integer arrays (values < 2^32); returns the four
    output words as uint64 arrays holding 32-bit values.
    """
    x = [np.asarray(c, dtype=np.uint64) & _MASK for c in (c0, c1, c2, c3)]
    x = list(np.broadcast_arrays(*x))
    ka = int(k0) & 0xFFFFFFFF
    kb = int(k1) & 0xFFFFFFFF
    for rnd in range(10):
        if rnd:
            ka = (ka + _W0) & 0xFFFFFFFF
            kb = (kb + _W1) & 0xFFFFFFFF
        hi0, lo0 = _mulhilo(_M0, x[0])
        hi1, lo1 = _mulhilo(_M1, x[2])
        x = [hi1 ^ x[1] ^ np.uint64(ka), lo1, hi0 ^ x[3] ^ np.uint64(kb), lo0]
    return x


def _words(seed: int, n: int, k: int, tag: int):
    """Output words w[i, j] for the n x k matrix (counter (i, j//4, tag, 0))."""
    nb = (k + 3) // 4
    i = np.arange(n, dtype=np.uint64)[:, None]
    b = np.arange(nb, dtype=np.uint64)[None, :]
    w = philox4x32_10(i, b, np.uint64(tag), np.uint64(0), seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    out = np.empty((n, nb * 4), dtype=np.uint64)
    for q in range(4):
        out[:, q::4] = w[q]
    return out[:, :k]


def omega_gaussian(seed: int, n: int, k: int) -> np.ndarray:
    """Gaussian Omega, Omega_ij ~ N(0, 1) (Sec. I-A), as FP32 values in FP64.

    Box-Muller: z_cos = sqrt(-2 ln u_a) cos(2 pi u_b), z_sin = ... sin(...),
    with (u_a, u_b) from the word pair (w0, w1) or (w2, w3).
    """
    w = _words(seed, n, ((k + 3) // 4) * 4, TAG_GAUSSIAN).astype(np.float64)
    u = (w + 0.5) * 2.0 ** -32
    out = np.empty_like(u)
    for a in (0, 2):
        ua = u[:, a::4]
        ub = u[:, a + 1::4]
        rad = np.sqrt(-2.0 * np.log(ua))
        out[:, a::4] = rad * np.cos(2.0 * np.pi * ub)
        out[:, a + 1::4] = rad * np.sin(2.0 * np.pi * ub)
    return out[:, :k].astype(np.float32).astype(np.float64)


def sparse_threshold(p: int) -> int:
    """T = floor(2^32 / (2p)): P(w < T) = T / 2^32 ~ 1/(2p) (Sec. I-A)."""
    return (1 << 32) // (2 * int(p))


def omega_sparse(seed: int, n: int, k: int, p: int) -> np.ndarray:
    """Very sparse Omega in {-1, 0, +1} w.p. {1/2p, 1-1/p, 1/2p} (Sec. I-A)."""
    w = _words(seed, n, k, TAG_SPARSE)
    t = np.uint64(sparse_threshold(p))
    out = np.zeros(w.shape, dtype=np.float64)
    out[w < t] = -1.0
    out[(w >= t) & (w < 2 * t)] = 1.0
    return out


def bf16_rne(x: np.ndarray) -> np.ndarray:
    """Round FP64 -> FP32 (nearest-even) -> BF16 (nearest-even); FP64 result.

    The operand rounding the BF16 paths apply to Omega; not part of the
    method, only of its number format.
    """
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    lsb = (bits >> np.uint64(16)) & np.uint64(1)
    rounded = ((bits + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)
