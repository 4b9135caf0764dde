"""Counter-based splitmix64 random stream.

splitmix64 (Steele, Lea & Flood, OOPSLA 2014) is a bijective 64-bit mixer;
feeding it an incrementing counter gives a stream whose i-th value depends only
on (seed, i).  Uniforms take the top 53 bits; normals come from the
Box-Muller transform.  Everything is vectorised numpy on uint64 arrays, so a
million draws cost milliseconds and are identical on every host.
"""

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x):
    """Finaliser of splitmix64 applied elementwise to a uint64 array."""
    z = np.asarray(x, dtype=np.uint64).copy()
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Stream:
    """Random stream keyed by an integer seed and an optional tag.

    The tag separates independent streams drawn from one seed (for example
    the weights of different layers).  Successive calls continue the counter.
    """

    def __init__(self, seed, tag=0):
        key = np.array([(int(seed) * 0x100000001B3 + int(tag) * 0x9E3779B1)
                        & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
        self._key = splitmix64(key)[0]
        self._ctr = 0

    def u64(self, n):
        n = int(n)
        i = np.arange(self._ctr + 1, self._ctr + n + 1, dtype=np.uint64)
        self._ctr += n
        with np.errstate(over="ignore"):
            return splitmix64(self._key + i * _GOLDEN)

    def uniform(self, n, lo=0.0, hi=1.0):
        """n doubles uniform in [lo, hi) (53-bit resolution)."""
        u = (self.u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        return lo + (hi - lo) * u

    def normal(self, n, mean=0.0, std=1.0):
        """n standard-normal doubles by Box-Muller (one pair per two draws)."""
        m = (int(n) + 1) // 2
        u1 = self.uniform(m)
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log1p(-u1))      # 1-u1 in (0, 1]
        t = 2.0 * np.pi * u2
        z = np.concatenate([r * np.cos(t), r * np.sin(t)])[: int(n)]
        return mean + std * z
