"""Counter-based random draws for the cross's sampling step (oracle side).

The paper does not say how the random sample set of Alg. 2 is drawn; both the
oracle and the CUDA path use SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), each implemented from that
published definition.  SplitMix64 seeded with state s returns, as its m-th
output (m = 1, 2, ...), mix(s + m * GAMMA) with

    mix(z): z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27;
            z *= 0x94D049BB133111EB; z ^= z >> 31      (all mod 2^64)

A draw keyed by (seed, stream, counter) chains three such generators:
    s1   = first output of SplitMix64(seed)
    s2   = (stream + 1)-th output of SplitMix64(s1)
    draw = (counter + 1)-th output of SplitMix64(s2)
and a draw is mapped to an index in [0, M) by the high half of the 128-bit
product draw * M.
"""

MASK = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15

# stream purposes
PURPOSE_INIT = 0
PURPOSE_SAMPLE = 1


def mix(z: int) -> int:
    z &= MASK
    z ^= z >> 30
    z = (z * 0xBF58476D1CE4E5B9) & MASK
    z ^= z >> 27
    z = (z * 0x94D049BB133111EB) & MASK
    z ^= z >> 31
    return z


def splitmix_output(state: int, m: int) -> int:
    """m-th output (m >= 1) of SplitMix64 started from `state`."""
    return mix((state + m * GAMMA) & MASK)


def stream_id(sweep: int, k: int, purpose: int) -> int:
    """Stream for one (sweep, interface, purpose): sweep in the high 32 bits."""
    return ((sweep & 0xFFFFFFFF) << 32) | ((k & 0xFFFFFF) << 8) | (purpose & 0xFF)


def draw(seed: int, stream: int, counter: int) -> int:
    s1 = splitmix_output(seed & MASK, 1)
    s2 = splitmix_output(s1, (stream + 1) & MASK)
    return splitmix_output(s2, (counter + 1) & MASK)


def draw_index(seed: int, stream: int, counter: int, M: int) -> int:
    """Index in [0, M): floor(draw * M / 2^64)."""
    return (draw(seed, stream, counter) * M) >> 64
