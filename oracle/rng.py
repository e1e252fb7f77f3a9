"""SplitMix64 as a counter-based generator.

Published definition: Steele, Lea, Flood, "Fast splittable pseudorandom number
generators" (OOPSLA 2014); output function with the constants of Vigna's
public-domain ``splitmix64``.  The k-th output of a generator started at state
``s`` is ``mix(s + (k+1)*GAMMA)`` (mod 2^64), so any element can be computed
independently.  The method draws random numbers in two places: the initial
test vectors (Section 4.2, "r independent, random initial vectors") and the
priorities of the greedy independent-set coarsening.

Streams used here (counter = stream * 2^32 + i):
  V test vector k  -> stream 2k
  U test vector k  -> stream 2k + 1
  MIS priorities on level l -> stream 4096 + l
  colouring priorities on level l -> stream 6144 + l
"""
import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)


def mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
    return z ^ (z >> np.uint64(31))


def draw(seed: int, stream: int, count: int) -> np.ndarray:
    """uint64 outputs for counters stream*2^32 + i, i = 0..count-1."""
    ctr = (np.uint64(stream) << np.uint64(32)) + np.arange(count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed) + (ctr + np.uint64(1)) * GAMMA
    return mix(state)


def uniform_pm1(seed: int, stream: int, count: int) -> np.ndarray:
    """Uniform(-1, 1) doubles: 53 high bits scaled to [0,1), then 2u - 1."""
    u = (draw(seed, stream, count) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return 2.0 * u - 1.0


def initial_test_vectors(seed: int, n: int, r: int):
    """n x r blocks V (all random) and U (first column = 1, rest random).

    Section 4.2 starts from r random vectors for B and for B^T; Section 5 puts
    the known left null vector u^(1) = 1 in the U set.
    """
    V = np.empty((n, r))
    U = np.empty((n, r))
    for k in range(r):
        V[:, k] = uniform_pm1(seed, 2 * k, n)
        U[:, k] = uniform_pm1(seed, 2 * k + 1, n)
    U[:, 0] = 1.0
    return U, V
