"""Counter-based SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) - oracle side.

The paper leaves every random draw unspecified (random search vectors,
Sec. 3.1 step 4; disorder V_n of Eq. Ham; KPM probe vectors).  Both the oracle
and the CUDA library therefore implement one published generator from its
definition.  The generator started from state ``s`` returns, as its i-th output
(i = 0, 1, ...), ``mix64(s + (i + 1) * GAMMA)``; this module evaluates that
i-th output directly.  The starting state of a (seed, stream) pair is
``seed * 256 + stream``.

Streams: 0 = disorder potential, 1 = search vectors, 2 = KPM probe vectors,
3 = refill vectors of the orthonormalisation.
"""
import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

STREAM_DISORDER = 0
STREAM_SEARCH = 1
STREAM_KPM = 2
STREAM_REFILL = 3


def mix64(z):
    """SplitMix64 finaliser on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def words(seed, stream, index):
    """i-th SplitMix64 output of the generator started at seed*256+stream."""
    state = np.uint64((int(seed) * 256 + int(stream)) % (1 << 64))
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = state + (idx + np.uint64(1)) * GAMMA
    return mix64(z)


def uniform(seed, stream, index):
    """Uniform double in [0, 1): top 53 bits of the word times 2^-53 (exact)."""
    w = words(seed, stream, index)
    return (w >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
