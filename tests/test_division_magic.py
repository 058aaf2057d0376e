"""The multiply form of x / G used by the search kernels (div_magic in
hs_device.cuh, after Granlund and Montgomery's division by invariant
integers): with M = ceil(2^48 / G), floor(x M / 2^48) = floor(x / G) for every
x < 2^48 / G.  Checked here with exact integers at the edges of each residue
class, near the bound, and at random, for meshes from 2 to 65535 cells."""
import random


def magic(G):
    return -(-(1 << 48) // G)


def test_multiply_form_equals_division():
    rng = random.Random(11)
    for G in [2, 3, 5, 7, 250, 255, 1000, 1987, 2520, 4095, 5000, 20000, 65521, 65535]:
        M = magic(G)
        bound = (1 << 48) // G          # x < 2^48 / G
        xs = [0, 1, G - 1, G, G + 1, bound - 1, bound - G, bound - G - 1]
        xs += [q * G + r for q in (1, 10**6, bound // G - 1) for r in (0, G - 1)]
        xs += [rng.randrange(bound) for _ in range(2000)]
        for x in xs:
            if 0 <= x < bound:
                assert (x * M) >> 48 == x // G, (G, x)
        # the kernels multiply by M << 16 and keep the high 64 bits
        assert (M << 16) < (1 << 64)
        for x in xs[:50]:
            if 0 <= x < bound:
                assert (x * (M << 16)) >> 64 == x // G


def test_bound_is_needed():
    """Past the bound the form can fail: for G = 3 (e = 2) a large x shows it."""
    G = 3
    M = magic(G)
    x = (1 << 49) - 1                   # far past 2^48 / 3
    assert (x * M) >> 48 != x // G
