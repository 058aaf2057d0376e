"""Width-generic statement of the sketch's hash family (TEST INFRASTRUCTURE ONLY).

Vector multiply-shift (Thorup 2015, "High Speed Hashing for Integers and
Strings", arXiv:1504.06804, the strongly universal vector scheme): for a key
x = (x_0 .. x_{d-1}) with x_i < 2^w, multipliers a_i and increment b drawn from
[2^wbar), the l-bit hash

    h(x) = ((sum_i a_i * x_i + b) mod 2^wbar) >> (wbar - l)

is strongly universal (pairwise independent and uniform) when
wbar >= w + l - 1.  The Count Sketch needs a 2-independent bucket hash and a
2-independent sign hash per row (arXiv:1711.00975, Sec. 2.2); one l-bit hash
with l = log2(W) + 1 supplies both: the top log2(W) bits are the bucket and the
next bit is the sign (1 -> -1).

The sketch uses wbar = 64 and three 32-bit cell coordinates; tests run this
function at tiny widths, where strong universality can be checked by
enumerating every (a, b), and at wbar = 64 against the C oracle.
"""
from __future__ import annotations

import numpy as np


def multiply_shift(x, a, b: int, wbar: int, l: int) -> int:
    """l-bit vector multiply-shift of integer vector x (Python big ints)."""
    assert len(x) == len(a) and 1 <= l <= wbar
    v = b
    for xi, ai in zip(x, a):
        v += int(ai) * int(xi)
    v &= (1 << wbar) - 1
    return v >> (wbar - l)


def bucket_sign(x, a, b: int, log2w: int, wbar: int = 64) -> tuple[int, int]:
    """(bucket, sign) split of the (log2w + 1)-bit hash."""
    h = multiply_shift(x, a, b, wbar, log2w + 1)
    return h >> 1, (-1 if (h & 1) else 1)


def multiply_shift_table(xs: np.ndarray, wbar: int, l: int) -> np.ndarray:
    """Hash of every key in xs (shape (m, d)) under EVERY (a_0..a_{d-1}, b) in
    [2^wbar)^(d+1); returns an (m, 2^(wbar*(d+1))) table (small widths only)."""
    xs = np.asarray(xs, np.int64)
    m, d = xs.shape
    q = 1 << wbar
    grids = np.meshgrid(*([np.arange(q, dtype=np.int64)] * (d + 1)), indexing="ij")
    flat = [g.ravel() for g in grids]
    out = np.empty((m, q ** (d + 1)), np.int64)
    for i in range(m):
        v = flat[d].copy()
        for j in range(d):
            v += flat[j] * xs[i, j]
        out[i] = (v & (q - 1)) >> (wbar - l)
    return out
