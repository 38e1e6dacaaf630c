"""Counter-based probe generator (oracle side; test infrastructure only).

Algorithm 3 step 2 draws a Rademacher (or Gaussian) sketch S, and step 6 draws further random
vectors G. The paper uses NumPy's stream, which cannot and need not be reproduced; this library
defines its probes by a counter-based generator so that the GPU and the oracle draw identical
vectors without sharing code. Each side implements this definition on its own.

  mix(z)   = SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014) applied to
             z + 0x9E3779B97F4A7C15, i.e. the first output of SplitMix64 seeded with z:
               z += 0x9E3779B97F4A7C15
               z  = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
               z  = (z ^ (z >> 27)) * 0x94D049BB133111EB
               return z ^ (z >> 31)                      (all mod 2^64)
  counter  = stream * 2^56 + col * 2^32 + row            (row < 2^32, col < 2^24)
  x        = mix(seed XOR mix(counter))
  Rademacher: +1 if the top bit of x is 0, else -1.
  Gaussian:   u1 = ((x >> 11) + 1) * 2^-53,  u2 = (mix(x) >> 11) * 2^-53,
              g  = sqrt(-2 ln u1) * cos(2 pi u2)         (Box-Muller).
Streams: 0 = S (sketch), 1 = G (residual probes), 2 = power-iteration start vector.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)

STREAM_S = 0
STREAM_G = 1
STREAM_POWER = 2


def mix(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + GOLDEN
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
    return z ^ (z >> np.uint64(31))


def raw_bits(seed: int, stream: int, n: int, cols: int, col0: int = 0) -> np.ndarray:
    """x[row, col] = mix(seed XOR mix(counter)) as an (n, cols) uint64 array."""
    rows = np.arange(n, dtype=np.uint64)[:, None]
    cc = np.arange(col0, col0 + cols, dtype=np.uint64)[None, :]
    ctr = (np.uint64(stream) << np.uint64(56)) | (cc << np.uint64(32)) | rows
    return mix(np.uint64(seed) ^ mix(ctr))


def rademacher(seed: int, stream: int, n: int, cols: int) -> np.ndarray:
    x = raw_bits(seed, stream, n, cols)
    return np.where((x >> np.uint64(63)) == 0, 1.0, -1.0)


def gaussian(seed: int, stream: int, n: int, cols: int) -> np.ndarray:
    x = raw_bits(seed, stream, n, cols)
    u1 = ((x >> np.uint64(11)) + np.uint64(1)).astype(np.float64) * 2.0 ** -53
    u2 = (mix(x) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def probes(kind: str, seed: int, stream: int, n: int, cols: int) -> np.ndarray:
    if kind == "rademacher":
        return rademacher(seed, stream, n, cols)
    if kind == "gaussian":
        return gaussian(seed, stream, n, cols)
    raise ValueError(kind)
