"""SplitMix64 counter-based generator (Steele, Lea and Flood, OOPSLA 2014).

The state advances by the golden-ratio increment 0x9E3779B97F4A7C15 and each
output is the state passed through the published 64-bit finaliser
(xor-shift 30, multiply 0xBF58476D1CE4E5B9, xor-shift 27, multiply
0x94D049BB133111EB, xor-shift 31).  Doubles in [0, 1) take the top 53 bits.
Because the n-th output depends only on seed + n*increment, the stream can be
produced vectorised with numpy's wrapping uint64 arithmetic.
"""
import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _finalise(z):
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64_stream(seed, count, start=0):
    """Outputs start .. start+count-1 of the stream seeded with `seed` (uint64)."""
    with np.errstate(over="ignore"):
        n = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + n * _GAMMA
        return _finalise(state)


class SplitMix64:
    """Sequential view of the stream: each draw consumes the next outputs."""

    def __init__(self, seed):
        self.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
        self.pos = 0

    def next_u64(self, count):
        out = splitmix64_stream(self.seed, count, self.pos)
        self.pos += count
        return out

    def uniform(self, count, lo=0.0, hi=1.0):
        """`count` doubles uniform in [lo, hi) from the top 53 bits of each output."""
        u = (self.next_u64(count) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u
