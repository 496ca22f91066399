"""Counter-based random numbers for the synthetic inputs.

The generator is SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used in its counter form: the
k-th output of a stream is the SplitMix64 output function applied to
``base + (k + 1) * GAMMA`` (arithmetic mod 2^64).  Because every output
depends only on (seed, stream id, counter), a whole array is produced with
vectorised uint64 arithmetic and the values are identical on every machine
and every numpy version.

Doubles in [0, 1) take the top 53 bits of an output.  Normals use the
Box-Muller transform.  Poisson counts use sequential-search inversion of
the cumulative distribution (Devroye, "Non-Uniform Random Variate
Generation", 1986, Sec. X.3.3), vectorised over the array; binomial counts
by the same inversion with the ratio of successive probabilities.

This module only draws numbers; it holds none of the INLA method.
"""
import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z):
    """SplitMix64 output function (the 'mix64variant13' finaliser)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


class Stream:
    """One independent substream, identified by (seed, stream_id).

    Successive calls continue the counter, so ``s.uniform(3); s.uniform(2)``
    returns the same five numbers as ``s.uniform(5)``.
    """

    def __init__(self, seed: int, stream_id: int):
        with np.errstate(over="ignore"):
            key = _mix(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ (np.uint64(stream_id) * GAMMA))
            self.base = np.uint64(_mix(key + np.uint64(0x632BE59BD9B4E019)))
        self.counter = 0

    def bits(self, n: int) -> np.ndarray:
        k = np.arange(self.counter + 1, self.counter + 1 + n, dtype=np.uint64)
        self.counter += n
        with np.errstate(over="ignore"):
            return _mix(self.base + k * GAMMA)

    def uniform(self, n: int) -> np.ndarray:
        """n doubles in [0, 1)."""
        return (self.bits(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def uniform_open(self, n: int) -> np.ndarray:
        """n doubles in (0, 1), for logarithms."""
        return ((self.bits(n) >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)

    def integers(self, n: int, high: int) -> np.ndarray:
        """n integers uniform on {0, ..., high-1} (multiply-shift on 32 bits)."""
        top = (self.bits(n) >> np.uint64(32)).astype(np.uint64)
        return ((top * np.uint64(high)) >> np.uint64(32)).astype(np.int64)

    def normal(self, n: int) -> np.ndarray:
        """n standard normals by Box-Muller (both outputs of each pair used)."""
        h = (n + 1) // 2
        u1 = self.uniform_open(h)
        u2 = self.uniform(h)
        r = np.sqrt(-2.0 * np.log(u1))
        out = np.empty(2 * h)
        out[0::2] = r * np.cos(2.0 * np.pi * u2)
        out[1::2] = r * np.sin(2.0 * np.pi * u2)
        return out[:n]

    def poisson(self, mean: np.ndarray) -> np.ndarray:
        """Poisson counts with the given means by CDF inversion.

        Each count uses one uniform.  Means above 700 would underflow exp(-mean)
        and are rejected (the synthetic workloads stay far below).
        """
        mean = np.asarray(mean, dtype=np.float64)
        if mean.size and float(mean.max()) > 700.0:
            raise ValueError("poisson: mean too large for inversion")
        u = self.uniform(mean.size)
        k = np.zeros(mean.size, dtype=np.int64)
        p = np.exp(-mean)
        cdf = p.copy()
        active = u > cdf
        while np.any(active):
            idx = np.nonzero(active)[0]
            k[idx] += 1
            p[idx] *= mean[idx] / k[idx]
            cdf[idx] += p[idx]
            # stop when the cdf passes u, or when the tail has vanished in rounding
            active[idx] = (u[idx] > cdf[idx]) & (p[idx] > 0.0)
        return k

    def negbinomial(self, size: int, mean: np.ndarray) -> np.ndarray:
        """Negative binomial counts NB(mean, size) for an integer size r: the sum of r
        geometric counts of success probability r / (r + mean), each by inversion
        floor(log U / log(1 - p)) of one uniform (r uniforms per count)."""
        mean = np.asarray(mean, dtype=np.float64)
        q = mean / (size + mean)                    # failure probability 1 - p
        u = self.uniform_open(size * mean.size).reshape(size, mean.size)
        with np.errstate(divide="ignore"):
            g = np.floor(np.log(u) / np.log(q))
        g = np.where(q > 0.0, g, 0.0)
        return g.sum(axis=0).astype(np.int64)

    def binomial(self, trials: np.ndarray, p: np.ndarray) -> np.ndarray:
        """Binomial counts Bin(trials, p) by CDF inversion, one uniform each."""
        n = np.asarray(trials, dtype=np.int64)
        p = np.asarray(p, dtype=np.float64)
        q = 1.0 - p
        u = self.uniform(n.size)
        k = np.zeros(n.size, dtype=np.int64)
        pk = q ** n
        cdf = pk.copy()
        active = (u > cdf) & (k < n)
        while np.any(active):
            idx = np.nonzero(active)[0]
            pk[idx] *= (n[idx] - k[idx]) / (k[idx] + 1.0) * (p[idx] / q[idx])
            k[idx] += 1
            cdf[idx] += pk[idx]
            active[idx] = (u[idx] > cdf[idx]) & (k[idx] < n[idx])
        return k
