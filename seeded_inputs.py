"""Seeded synthetic inputs for the CKKS key-switching path.

This module is shared by the CPU oracle, the tests and the benchmark.  It holds
sampling only: no transform, no base conversion and no modular product of the
method lives here.  Everything the method computes is done independently by the
oracle (``oracle/``) and by the CUDA library (``paper_2507_04775_gb300/``).

Generator
---------
SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) used as a counter-based generator: word ``i`` of a
stream keyed by ``key`` is ``mix64(key + (i + 1) * GAMMA)`` with GAMMA the
golden-ratio increment 0x9E3779B97F4A7C15 and ``mix64`` the published
finaliser.  Because every word is a pure function of (key, i), numpy can
generate millions of words at once and the result does not depend on how the
work is split.

Distributions (the recipe of the synthetic workload)
----------------------------------------------------
* ``uniform_mod(q, n)``   -- uniform residues in [0, q) by rejection sampling on
  the top ``bitlen(q)`` bits of each word (accepted words kept in order).
* ``ternary(n)``          -- uniform on {-1, 0, 1} (rejection on 2-bit values).
* ``sparse_ternary(n, h)``-- exactly ``h`` non-zeros at positions chosen by a
  partial Fisher-Yates shuffle, each +1 or -1 with probability 1/2.
* ``gaussian(n, sigma)``  -- Box-Muller normal in FP64, rounded half away from
  zero, samples beyond 6 sigma rejected; sigma = 3.2 by default.
* ``uniform_real(n)``     -- FP64 uniform on [-1, 1) with 53 random bits.
* ``complex_slots(n)``    -- real and imaginary parts independently uniform on
  [-1, 1).

Streams are named by small integers so that, e.g., the secret and the
encryption randomness of one workload never overlap.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64_int(z: int) -> int:
    """SplitMix64 finaliser on a Python int (used to derive stream keys)."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def _mix64_np(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser on a uint64 array (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Stream:
    """A counter-based SplitMix64 stream.

    ``Stream(seed, stream_id)`` is fully determined by its two integers; every
    draw advances an internal word counter so successive calls never reuse a
    word.
    """

    def __init__(self, seed: int, stream_id: int = 0):
        self.key = _mix64_int((seed & MASK64) ^ _mix64_int(stream_id * GAMMA + 1))
        self.counter = 0

    def words(self, n: int) -> np.ndarray:
        """``n`` raw 64-bit words."""
        idx = np.arange(self.counter + 1, self.counter + 1 + n, dtype=np.uint64)
        self.counter += n
        with np.errstate(over="ignore"):
            z = np.uint64(self.key) + idx * np.uint64(GAMMA)
        return _mix64_np(z)

    # -- integers ---------------------------------------------------------
    def uniform_mod(self, q: int, n: int) -> np.ndarray:
        """``n`` residues uniform in [0, q), q < 2^63, by rejection."""
        bits = int(q - 1).bit_length()
        out = np.empty(n, dtype=np.uint64)
        filled = 0
        while filled < n:
            want = n - filled
            # acceptance probability is > 1/2, draw a little more than twice
            w = self.words(2 * want + 64) >> np.uint64(64 - bits)
            w = w[w < np.uint64(q)]
            take = min(want, w.size)
            out[filled:filled + take] = w[:take]
            filled += take
        return out

    def ternary(self, n: int) -> np.ndarray:
        """``n`` values uniform on {-1, 0, 1} as int64."""
        out = np.empty(n, dtype=np.int64)
        filled = 0
        while filled < n:
            want = n - filled
            w = (self.words(2 * want + 64) >> np.uint64(62)).astype(np.int64)
            w = w[w < 3]
            take = min(want, w.size)
            out[filled:filled + take] = w[:take] - 1
            filled += take
        return out

    def below(self, bound: int) -> int:
        """One integer uniform in [0, bound) by rejection."""
        bits = max(1, int(bound - 1).bit_length())
        while True:
            v = int(self.words(1)[0]) >> (64 - bits)
            if v < bound:
                return v

    def sparse_ternary(self, n: int, h: int) -> np.ndarray:
        """Exactly ``h`` non-zero entries in {-1, 1}; positions by partial
        Fisher-Yates, signs uniform."""
        if not 0 <= h <= n:
            raise ValueError("hamming weight out of range")
        perm = np.arange(n, dtype=np.int64)
        for i in range(h):
            j = i + self.below(n - i)
            perm[i], perm[j] = perm[j], perm[i]
        out = np.zeros(n, dtype=np.int64)
        signs = self.words(h) >> np.uint64(63)
        out[perm[:h]] = np.where(signs == 1, -1, 1)
        return out

    # -- floating point ---------------------------------------------------
    def unit(self, n: int) -> np.ndarray:
        """``n`` FP64 values uniform in [0, 1) (53 random bits each)."""
        return (self.words(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def uniform_real(self, n: int) -> np.ndarray:
        """``n`` FP64 values uniform in [-1, 1)."""
        return 2.0 * self.unit(n) - 1.0

    def complex_slots(self, n: int) -> np.ndarray:
        """``n`` complex slots, real and imaginary parts uniform in [-1, 1)."""
        re = self.uniform_real(n)
        im = self.uniform_real(n)
        return re + 1j * im

    def gaussian(self, n: int, sigma: float = 3.2) -> np.ndarray:
        """Rounded Gaussian (Box-Muller, FP64), rejected beyond 6 sigma, int64."""
        out = np.empty(n, dtype=np.int64)
        filled = 0
        while filled < n:
            want = n - filled
            m = want // 2 + 32
            u1 = 1.0 - self.unit(m)          # (0, 1]
            u2 = self.unit(m)
            r = np.sqrt(-2.0 * np.log(u1))
            z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)]) * sigma
            z = z[np.abs(z) <= 6.0 * sigma]
            z = np.sign(z) * np.floor(np.abs(z) + 0.5)
            take = min(want, z.size)
            out[filled:filled + take] = z[:take].astype(np.int64)
            filled += take
        return out


# -- workload helpers ------------------------------------------------------

def uniform_poly(stream: Stream, primes, N: int) -> np.ndarray:
    """A limb-major ``[len(primes)][N]`` array of uniform residues, limb ``i``
    uniform mod ``primes[i]``."""
    out = np.empty((len(primes), N), dtype=np.uint64)
    for i, q in enumerate(primes):
        out[i] = stream.uniform_mod(int(q), N)
    return out


def workload_seed(config_index: int) -> int:
    """Seed of the synthetic workload with the given index (0..4)."""
    return 0xF1DE5000 + config_index


# -- parameter sets of the synthetic workloads --------------------------------
# Only the requests (ring degree, prime sizes and counts, digits) live here;
# each implementation finds its own primes from them.

@dataclass(frozen=True)
class ParamSet:
    name: str
    logN: int
    nq: int           # number of q-primes (ciphertext limbs at the top level)
    q_bits: int
    nk: int           # number of special primes
    p_bits: int
    dnum: int
    log_scale: int


# HMult+relin of one pair: N=4096, 3 x 40-bit q, 1 x 50-bit p, dnum=3, scale 2^40
SMALL = ParamSet("logN12-L3-K1-dnum3", 12, 3, 40, 1, 50, 3, 40)
# single-op path: N=65536, 30 x 54-bit q, 10 x 60-bit p, dnum=3, scale 2^40
FULL = ParamSet("logN16-L30-K10-dnum3", 16, 30, 54, 10, 60, 3, 40)
# a mid-size set for fast checks that still spans several digits and tiles
MID = ParamSet("logN12-L12-K4-dnum3", 12, 12, 54, 4, 60, 3, 40)
# the most primes a context takes (L + K = 64): digits of 16 limbs and 16 special primes
WIDE = ParamSet("logN12-L48-K16-dnum3", 12, 48, 54, 16, 60, 3, 40)
