"""Seeded synthetic input generators.

This module is the only code shared by the CUDA path, the benchmark and the
CPU oracle. It holds no arithmetic of the method (no NTT, no modular
multiplication, no key switching): it only draws random words and shapes them
into the value distributions of the paper's workloads:

* uniform residues in [0, q) for polynomial limbs and ciphertexts,
* ternary values in {-1, 0, 1} (secret key, encryption randomness),
* rounded Gaussian errors (sigma = 3.2, |e| < 20),
* complex message slots uniform in [-1, 1] x [-1, 1].

The generator is SplitMix64 (Steele, Lea and Flood, OOPSLA 2014; the public
domain reference by S. Vigna) used in its counter form: output number i of a
stream with key k is mix(k + (i + 1) * 0x9E3779B97F4A7C15), where mix is the
SplitMix64 finaliser. Being counter based, it vectorises in numpy and every
draw is a pure function of (seed, stream, counter).
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output finaliser, elementwise on uint64 (wrapping)."""
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _mix_scalar(x: int) -> int:
    return int(_mix(np.array([x & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0])


class Rng:
    """A SplitMix64 stream. Draws consume consecutive counters, so the values
    depend only on the seed and on the order of the calls."""

    def __init__(self, seed: int, stream: int = 0):
        # Stream key: the SplitMix64 finaliser of the (seed, stream) pair, so
        # that streams of one seed do not overlap in practice.
        self.key = np.uint64(_mix_scalar((seed * 0x9E3779B97F4A7C15 + stream) ^ 0xD1B54A32D192ED03))
        self.counter = 0

    def words(self, n: int) -> np.ndarray:
        """n raw 64-bit words."""
        idx = np.arange(self.counter + 1, self.counter + 1 + n, dtype=np.uint64)
        self.counter += n
        with np.errstate(over="ignore"):
            return _mix(self.key + idx * _GAMMA)

    def uniform_mod(self, q: int, n: int) -> np.ndarray:
        """n values uniform in [0, q) by rejection on the low bit_length(q) bits."""
        q = int(q)
        if q < 1:
            raise ValueError("q must be positive")
        bits = q.bit_length()
        mask = np.uint64((1 << bits) - 1) if bits < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
        out = np.empty(n, dtype=np.uint64)
        filled = 0
        while filled < n:
            need = n - filled
            draw = self.words(need + need // 2 + 64) & mask
            ok = draw[draw < np.uint64(q)]
            take = min(len(ok), need)
            out[filled:filled + take] = ok[:take]
            filled += take
        return out

    def uniform_limbs(self, moduli, n: int) -> np.ndarray:
        """[len(moduli)][n] array, row i uniform in [0, moduli[i])."""
        return np.stack([self.uniform_mod(int(q), n) for q in moduli]) if len(moduli) else \
            np.empty((0, n), dtype=np.uint64)

    def ternary(self, n: int) -> np.ndarray:
        """n int64 values uniform in {-1, 0, 1} (2-bit rejection sampling)."""
        out = np.empty(n, dtype=np.int64)
        filled = 0
        while filled < n:
            need = n - filled
            v = (self.words(need + need // 2 + 64) >> np.uint64(62)).astype(np.int64)
            v = v[v < 3]
            take = min(len(v), need)
            out[filled:filled + take] = v[:take] - 1
            filled += take
        return out

    def unit_doubles(self, n: int) -> np.ndarray:
        """n doubles uniform in [0, 1) from the top 53 bits."""
        return (self.words(n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))

    def gaussian(self, n: int, sigma: float = 3.2, bound: int = 20) -> np.ndarray:
        """n int64 values: a Box-Muller normal of deviation sigma rounded to the
        nearest integer, redrawn while |e| >= bound."""
        out = np.empty(n, dtype=np.int64)
        filled = 0
        while filled < n:
            need = n - filled
            m = need + 64
            u1 = self.unit_doubles(m)
            u2 = self.unit_doubles(m)
            r = np.sqrt(-2.0 * np.log1p(-u1))  # 1 - u1 in (0, 1]
            z = np.rint(sigma * r * np.cos(2.0 * np.pi * u2)).astype(np.int64)
            z = z[np.abs(z) < bound]
            take = min(len(z), need)
            out[filled:filled + take] = z[:take]
            filled += take
        return out

    def complex_slots(self, n: int) -> np.ndarray:
        """n complex values with real and imaginary parts uniform in [-1, 1)."""
        re = self.unit_doubles(n) * 2.0 - 1.0
        im = self.unit_doubles(n) * 2.0 - 1.0
        return re + 1j * im

    def choice(self, options, n: int) -> list:
        """n picks uniform over a short list (rejection on the low bits)."""
        k = len(options)
        bits = max(1, (k - 1).bit_length())
        out = []
        while len(out) < n:
            w = self.words(2 * (n - len(out)) + 8) & np.uint64((1 << bits) - 1)
            out.extend(options[int(x)] for x in w if int(x) < k)
        return out[:n]

    def exponential(self, n: int, rate: float) -> np.ndarray:
        """n inter-arrival gaps of a Poisson process with the given rate."""
        return -np.log1p(-self.unit_doubles(n)) / rate
