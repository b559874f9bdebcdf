"""SplitMix64 counter-based generator (oracle side).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

Sec. 2 ("Smoothers") starts the power method from a random vector at the first
Newton step.  That random vector is drawn inside the method, so both the
oracle and the CUDA library implement the same published generator
independently: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014).  Its state advances by the odd constant
GAMMA = 0x9E3779B97F4A7C15 and each output is the 64-bit finaliser

    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB
    z =  z ^ (z >> 31)

applied to the state.  Used as a counter-based generator, output number c
(c = 0, 1, ...) of the stream with key k is finaliser(k + (c + 1) * GAMMA).

Streams: key(seed, level) = seed + level * 0xD1B54A32D192ED03 (mod 2^64).
Counter: the linear index of the node in the full node grid (x fastest).
Value:   uniform on [-1, 1):  (z >> 11) * 2^-53 * 2 - 1.
Only interior nodes take a value; boundary nodes are 0.
"""
import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
LEVEL_MUL = np.uint64(0xD1B54A32D192ED03)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)


def finalise(z):
    """The SplitMix64 output function (Steele, Lea & Flood 2014) on uint64 z."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed, level):
    """Key of the power-method start stream of a level: seed + level * constant."""
    with np.errstate(over="ignore"):
        return np.uint64(seed) + np.uint64(level) * LEVEL_MUL


def uniform_pm1(seed, level, counters):
    """Uniform [-1,1) values for the given counters of stream (seed, level)."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = stream_key(seed, level) + (c + np.uint64(1)) * GAMMA
    z = finalise(z)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) * 2.0 - 1.0


def sequential(seed, count):
    """The plain sequential SplitMix64 stream from state=seed (for pinning the
    counter form against the published state-advancing form)."""
    out = []
    state = int(seed) & 0xFFFFFFFFFFFFFFFF
    for _ in range(count):
        state = (state + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
        z = z ^ (z >> 31)
        out.append(z)
    return out


def start_vector(shape, seed, level, mask=None):
    """Random power-method start vector on a full node grid of the given shape
    (counter = flat array index); zero where mask is False (default: the
    boundary nodes of a scalar grid)."""
    idx = np.arange(int(np.prod(shape)), dtype=np.uint64).reshape(shape)
    v = uniform_pm1(seed, level, idx)
    if mask is None:
        from .fem import boundary_mask
        v[boundary_mask(shape)] = 0.0
    else:
        v[~mask] = 0.0
    return v
