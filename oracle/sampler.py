"""Counter-based random draws for the initial column block J_1 (Alg. 1 line 1,
Alg. 2 line 1: "a random index set of cardinality d").

TEST INFRASTRUCTURE ONLY (see the package docstring).

The generator is SplitMix64 as published by Steele, Lea and Flood ("Fast
splittable pseudorandom number generators", OOPSLA 2014): the state advances
by the golden gamma 0x9E3779B97F4A7C15 and each output is the state passed
through the variant-13 mixing function
    z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31.

Stream of block ``b`` (a leaf or a batched block): initial state
    s_0 = seed XOR (b * 0xD1342543DE82EF95 mod 2^64).
Draw t (t = 0, 1, ...) is the (t+1)-th output of that stream.

J_1 of a leaf with n local columns: a partial Fisher-Yates shuffle of
[0, n): for t = 0 .. min(d, n)-1, j = t + ((z_t >> 32) * (n - t)) >> 32,
swap perm[t], perm[j]; J_1 = perm[0 : min(d, n)].
"""

MASK64 = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15
STREAM_MULT = 0xD1342543DE82EF95


def splitmix64_outputs(state, count):
    """Return ``count`` SplitMix64 outputs starting from ``state``."""
    out = []
    s = state & MASK64
    for _ in range(count):
        s = (s + GOLDEN_GAMMA) & MASK64
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        z = z ^ (z >> 31)
        out.append(z)
    return out


def stream_state(seed, block_id):
    """Initial state of the draw stream of block ``block_id``."""
    return (seed ^ ((block_id * STREAM_MULT) & MASK64)) & MASK64


def block_id(batch_index, leaf_row, leaf_col):
    """Stream id of leaf (leaf_row, leaf_col) of batched block ``batch_index``
    (``batch_index`` = 0 for a single H-BACA call)."""
    return (batch_index << 24) | (leaf_row << 12) | leaf_col


def initial_columns(seed, bid, n, d):
    """Random initial block J_1 (local column indices of a leaf with n columns)."""
    dd = min(d, n)
    z = splitmix64_outputs(stream_state(seed, bid), dd)
    perm = list(range(n))
    for t in range(dd):
        j = t + (((z[t] >> 32) * (n - t)) >> 32)
        perm[t], perm[j] = perm[j], perm[t]
    return perm[:dd]
