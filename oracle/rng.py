"""Oracle side of the counter-based random streams (FP64 / uint64, numpy).

TEST INFRASTRUCTURE ONLY: nothing in the product path may import this module.

The paper leaves the generators open. CountSketch (Sec. 3.4.3) needs a hash
h: [n] -> [r] and random signs; the Gaussian embeddings (Sec. 3.4.1) need
i.i.d. N(0,1) entries. This oracle draws all of them from the splitmix64
generator (Steele, Lea and Flood, OOPSLA 2014) used as a pure function of
(key, counter), so every entry depends only on the seed and its index:

* ``splitmix64(key, c)`` is the c-th output of splitmix64 started from state
  ``key``: state_c = key + (c+1) * 0x9E3779B97F4A7C15 (mod 2^64), followed by
  the published 64-bit finaliser (xor-shift 30, multiply 0xBF58476D1CE4E5B9,
  xor-shift 27, multiply 0x94D049BB133111EB, xor-shift 31).
* Stream keys: key_t = seed XOR (t * 0xD1B54A32D192ED03 mod 2^64), with
  t = 1 for the CountSketch hash, 2 for the Gaussian sketch G and 3 for the
  JL matrix Omega.
* Bucket and sign of row i: x = splitmix64(key_1, i); h(i) = (hi32(x) * s) >> 32
  (multiply-shift, no modulo bias); sigma_i = +1 if bit 0 of x is 0, else -1.
* Standard normal number c of stream t (Box-Muller, cosine branch only):
  u1 = ((splitmix64(key_t, 2c) >> 11) + 1) * 2^-53 in (0, 1],
  u2 = (splitmix64(key_t, 2c+1) >> 11) * 2^-53 in [0, 1),
  g = sqrt(-2 ln u1) * cos(2 pi u2).
* Entries of the Gaussian sketch G (stream 2): N_c / sqrt(m), the FP64 draw itself scaled as a
  Gaussian embedding (Sec. 3.4.1). The paper's G is Gaussian; no rounding of the draws is part of
  the method.

Reading note (the paper asks for 2-wise independent h and 4-wise independent
signs, Sec. 3.4.3): splitmix64 is not provably k-wise independent; it is used
as a counter-based hash so that the CPU and GPU sides can both evaluate it.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_MUL1 = np.uint64(0xBF58476D1CE4E5B9)
_MUL2 = np.uint64(0x94D049BB133111EB)
_STREAM_MUL = 0xD1B54A32D192ED03
STREAM_HASH, STREAM_G, STREAM_OMEGA = 1, 2, 3
STREAM_SRHT_SIGN, STREAM_SRHT_ROWS = 4, 5
_MASK64 = (1 << 64) - 1


def stream_key(seed: int, stream: int) -> int:
    """key_t = seed XOR (t * 0xD1B54A32D192ED03) mod 2^64."""
    return (int(seed) ^ ((stream * _STREAM_MUL) & _MASK64)) & _MASK64


def splitmix64(key: int, counter) -> np.ndarray:
    """c-th splitmix64 output from state ``key``, vectorised over ``counter``."""
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(key & _MASK64) + (c + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _MUL1
        z = (z ^ (z >> np.uint64(27))) * _MUL2
        z = z ^ (z >> np.uint64(31))
    return z


def bucket_and_sign(n: int, s: int, seed: int, start: int = 0):
    """CountSketch hash of rows start..start+n-1: (bucket int64, sign float64)."""
    assert 1 <= s < (1 << 32)
    x = splitmix64(stream_key(seed, STREAM_HASH), np.arange(start, start + n, dtype=np.uint64))
    b = ((x >> np.uint64(32)) * np.uint64(s)) >> np.uint64(32)
    sign = np.where((x & np.uint64(1)) == 0, 1.0, -1.0)
    return b.astype(np.int64), sign


def srht_signs(s: int, seed: int) -> np.ndarray:
    """Diagonal of D of the SRHT (Sec. 3.4.2): +1 / -1 from bit 0 of stream 4 at counters 0..s-1."""
    x = splitmix64(stream_key(seed, STREAM_SRHT_SIGN), np.arange(s, dtype=np.uint64))
    return np.where((x & np.uint64(1)) == 0, 1.0, -1.0)


def srht_rows(t: int, s: int, seed: int) -> np.ndarray:
    """Rows of P of the SRHT: t independent uniform draws from [0, s), multiply-shift of the high
    word of stream 5 at counters 0..t-1."""
    x = splitmix64(stream_key(seed, STREAM_SRHT_ROWS), np.arange(t, dtype=np.uint64))
    return (((x >> np.uint64(32)) * np.uint64(s)) >> np.uint64(32)).astype(np.int64)


def unit_open_closed(x) -> np.ndarray:
    """u in (0, 1] from a 64-bit word: ((x >> 11) + 1) 2^-53 (the u1 of Box-Muller, never 0)."""
    return ((np.asarray(x, dtype=np.uint64) >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53


def unit_closed_open(x) -> np.ndarray:
    """u in [0, 1) from a 64-bit word: (x >> 11) 2^-53 (the u2 of Box-Muller)."""
    return (np.asarray(x, dtype=np.uint64) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def gaussian(seed: int, stream: int, counters) -> np.ndarray:
    """Box-Muller standard normals (FP64) for the given counters of a stream: sqrt(-2 ln u1)
    cos(2 pi u2), cosine branch only (the generator definition of the random streams)."""
    c = np.asarray(counters, dtype=np.uint64)
    key = stream_key(seed, stream)
    with np.errstate(over="ignore"):
        x1 = splitmix64(key, np.uint64(2) * c)
        x2 = splitmix64(key, np.uint64(2) * c + np.uint64(1))
    u1 = unit_open_closed(x1)
    u2 = unit_closed_open(x2)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def sketch_gaussian(seed: int, counters, m: int) -> np.ndarray:
    """Entries of G by counter: N_c / sqrt(m), N_c the counter's Box-Muller draw (stream 2; the
    Gaussian embedding of Sec. 3.4.1 scaled by 1/sqrt(m))."""
    return gaussian(seed, STREAM_G, counters) / np.sqrt(m)


def gaussian_sketch_block(m: int, s: int, seed: int, c0: int, c1: int) -> np.ndarray:
    """Columns c0..c1-1 of G (m x s): G[j, b] = N_{j*s+b} / sqrt(m)."""
    j = np.arange(m, dtype=np.uint64)[:, None]
    b = np.arange(c0, c1, dtype=np.uint64)[None, :]
    with np.errstate(over="ignore"):
        idx = j * np.uint64(s) + b
    return sketch_gaussian(seed, idx, m)


def omega(r: int, k: int, seed: int) -> np.ndarray:
    """JL matrix Omega (r x k): Omega[p, q] = N_{p*k+q} / sqrt(k); p is the pivot position."""
    idx = np.arange(r * k, dtype=np.uint64).reshape(r, k)
    return gaussian(seed, STREAM_OMEGA, idx) / np.sqrt(k)
