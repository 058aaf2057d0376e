"""Pins of the CPU oracle against what the paper and mathematics fix.

Every check here compares the oracle with something other than itself:
published known-answer values, hand-derived fixtures, exhaustive enumeration
of the hash family at tiny widths, exact counts, brute force on tiny
dictionaries and statistical laws.
"""
import itertools
import math
from collections import Counter

import numpy as np
import pytest

import oracle
from oracle import hashref
from tests.conftest import golden_path


def _golden_rows(name):
    rows = []
    with open(golden_path(name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------- splitmix64

def test_splitmix64_known_answers():
    want = [int(r[1], 16) for r in _golden_rows("splitmix64_seed0.txt")]
    assert oracle.splitmix64_sequence(0, len(want)) == want
    for g, w in enumerate(want):
        assert oracle.splitmix64_at(0, g) == w


def test_row_seeds_are_the_splitmix_sequence():
    # row r takes outputs 4r..4r+3 as (a0, a1, a2, b)
    want = [int(r[1], 16) for r in _golden_rows("splitmix64_seed0.txt")]
    s = oracle.derive_seeds(0, 3)
    assert [int(v) for v in s[:4]] == want
    assert [int(v) for v in s] == oracle.splitmix64_sequence(0, 12)


def test_sampling_decisions_follow_the_published_sequence():
    # rate 0.5 -> threshold 2^63; keep iff the g-th output is below it
    want = [int(r[1], 16) for r in _golden_rows("splitmix64_seed0.txt")]
    assert oracle.sample_threshold(0.5) == 1 << 63
    for g, w in enumerate(want):
        assert oracle.keep(g, 0, 0.5) == (w < (1 << 63))
    # the first output 0xe220... is >= 2^63: particle 0 is dropped, 1 and 2 kept
    assert [oracle.keep(g, 0, 0.5) for g in range(3)] == [False, True, True]
    assert all(oracle.keep(g, 12345, 1.0) for g in range(100))
    assert oracle.sample_threshold(0.25) == 1 << 62


def test_sampling_rate_is_binomial():
    n = 200_000
    for rate in (0.5, 0.1, 1.0 / 16):
        kept = int(oracle.keep_mask(0, n, 77, rate).sum())
        sd = math.sqrt(n * rate * (1 - rate))
        assert abs(kept - n * rate) < 6 * sd
    # deterministic per index
    a = oracle.keep_mask(1000, 5000, 9, 0.1)
    b = oracle.keep_mask(1000, 5000, 9, 0.1)
    assert np.array_equal(a, b)


# -------------------------------------------------------------- quantisation

def test_quantisation_golden_cases():
    p = oracle.Params(5, 10, 100.0, 0.1, 0)
    assert p.G == 1000 and p.inv_cell == 10.0
    for r in _golden_rows("quantize_cases.txt"):
        x, y, z = (float(np.float32(v)) for v in r[:3])
        c = oracle.cell_of(x, y, z, p)
        assert c == tuple(int(v) for v in r[3:6]), r
        key = int(oracle.keys_of(np.array([[x, y, z]], np.float32), p)[0])
        assert key == int(r[6]), r


def test_quantisation_matches_float32_floor_on_random_points():
    # numpy float32 multiply is one IEEE rounding; floor then periodic wrap
    rng = np.random.default_rng(5)
    p = oracle.Params(5, 10, 100.0, 0.1, 0)
    xyz = rng.uniform(-150, 250, size=(20000, 3)).astype(np.float32)
    prod = (xyz * np.float32(p.inv_cell)).astype(np.float32)
    c = np.mod(np.floor(prod).astype(np.int64), p.G)
    want = c[:, 0] + p.G * (c[:, 1] + p.G * c[:, 2])
    assert np.array_equal(oracle.keys_of(xyz, p), want.astype(np.uint64))


def test_quantisation_skips_non_finite():
    p = oracle.Params(5, 10, 100.0, 0.1, 0)
    bad = np.array([[np.nan, 1, 1], [1, np.inf, 1], [1, 1, -np.inf], [1e30, 1, 1]], np.float32)
    assert np.all(oracle.keys_of(bad, p) == oracle.INVALID_KEY)


# ------------------------------------------------------------------- hashing

@pytest.mark.parametrize("xs", [((0, 0, 0), (1, 0, 0)), ((1, 2, 3), (3, 2, 1)),
                                ((0, 0, 1), (0, 1, 0)), ((3, 3, 3), (2, 3, 3))])
def test_multiply_shift_strongly_universal_exhaustive(xs):
    # wbar = 5-bit words, 2-bit coordinates, l = wbar - w + 1 = 4 output bits:
    # over all 2^20 (a0, a1, a2, b), every pair of outputs occurs equally often
    wbar, l = 5, 4
    tab = hashref.multiply_shift_table(np.array(xs), wbar, l)
    pair = tab[0] * (1 << l) + tab[1]
    counts = np.bincount(pair, minlength=1 << (2 * l))
    assert counts.min() == counts.max() == tab.shape[1] >> (2 * l)


def test_multiply_shift_without_increment_is_not_universal():
    # a mutated family (b dropped) must fail the same exhaustive check, so the
    # check above really constrains the formula
    wbar, l = 5, 4
    tab = hashref.multiply_shift_table(np.array([(0, 0, 0), (1, 0, 0)]), wbar, l)
    q = 1 << wbar
    no_b = tab[:, ::q]    # b = 0 slice
    pair = no_b[0] * (1 << l) + no_b[1]
    counts = np.bincount(pair, minlength=1 << (2 * l))
    assert counts.min() != counts.max()


def test_c_hash_equals_generic_statement():
    rng = np.random.default_rng(11)
    for log2w in (1, 8, 16, 24, 26, 30):
        p = oracle.Params(7, log2w, 500.0, 0.1, int(rng.integers(0, 2**63)))
        for _ in range(200):
            c3 = [int(v) for v in rng.integers(0, p.G, size=3)]
            r = int(rng.integers(0, p.rows))
            s = [int(v) for v in p.seeds[4 * r:4 * r + 4]]
            want = hashref.bucket_sign(c3, s[:3], s[3], log2w)
            assert oracle.hash_row(p, r, c3) == want


# -------------------------------------------------------------------- sketch

def _py_counters(p, keys):
    """Counters by the definition of Add, with the generic hash statement."""
    C = np.zeros((p.rows, p.width), np.int64)
    for key, f in Counter(int(k) for k in keys).items():
        c3 = oracle.key_decode(key, p.G)
        for r in range(p.rows):
            s = [int(v) for v in p.seeds[4 * r:4 * r + 4]]
            b, sg = hashref.bucket_sign(c3, s[:3], s[3], p.log2_width)
            C[r, b] += sg * f
    return C


def _box_points(rng, n, box, clusters=8):
    # clustered points so cells repeat
    centres = rng.uniform(0, box, size=(clusters, 3))
    pts = centres[rng.integers(0, clusters, n)] + rng.normal(0, box / 60, size=(n, 3))
    return np.mod(pts, box).astype(np.float32)


def test_sketch_equals_definition_of_add():
    rng = np.random.default_rng(3)
    p = oracle.Params(5, 6, 1.6, 0.1, 42)           # G = 16, W = 64: many collisions
    xyz = _box_points(rng, 3000, 1.6)
    C = oracle.sketch_update(oracle.new_counters(p), p, xyz)
    assert np.array_equal(C.astype(np.int64), _py_counters(p, oracle.keys_of(xyz, p)))


def test_exact_counts_at_large_width_without_collisions():
    rng = np.random.default_rng(4)
    p = oracle.Params(5, 24, 100.0, 0.1, 7)
    xyz = _box_points(rng, 8000, 100.0, clusters=40)
    keys = oracle.keys_of(xyz, p)
    exact = Counter(int(k) for k in keys)
    C = oracle.sketch_update(oracle.new_counters(p), p, xyz)
    # which (row, bucket) pairs are shared by two observed keys
    owners = {}
    for key in exact:
        for r in range(p.rows):
            b, _ = oracle.hash_row(p, r, oracle.key_decode(key, p.G))
            owners.setdefault((r, b), []).append(key)
    clean = 0
    for key, f in exact.items():
        rows = oracle.row_estimates(C, p, key)
        for r in range(p.rows):
            b, _ = oracle.hash_row(p, r, oracle.key_decode(key, p.G))
            if len(owners[(r, b)]) == 1:
                assert rows[r] == f
                clean += 1
        assert oracle.estimate(C, p, [key])[0] == f or any(
            len(owners[(r, oracle.hash_row(p, r, oracle.key_decode(key, p.G))[0])]) > 1
            for r in range(p.rows))
    assert clean > 0.99 * p.rows * len(exact)


def test_row_sum_invariant():
    rng = np.random.default_rng(8)
    p = oracle.Params(5, 12, 100.0, 0.1, 99, sample_seed=5)
    xyz = _box_points(rng, 20000, 100.0)
    for rate in (1.0, 0.3):
        C = oracle.sketch_update(oracle.new_counters(p), p, xyz, rate=rate)
        kept = oracle.keep_mask(0, len(xyz), p.sample_seed, rate)
        f = Counter(int(k) for k in oracle.keys_of(xyz[kept], p))
        for r in range(p.rows):
            s = [int(v) for v in p.seeds[4 * r:4 * r + 4]]
            want = sum(hashref.bucket_sign(oracle.key_decode(k, p.G), s[:3], s[3],
                                           p.log2_width)[1] * v for k, v in f.items())
            assert int(C[r].astype(np.int64).sum()) == want
            assert int(np.abs(C[r].astype(np.int64)).sum()) <= int(kept.sum())


def test_linearity_order_and_threads():
    rng = np.random.default_rng(9)
    p = oracle.Params(5, 10, 100.0, 0.1, 3, sample_seed=17)
    xyz = _box_points(rng, 30000, 100.0)
    whole = oracle.sketch_update(oracle.new_counters(p), p, xyz, rate=0.5)
    a = oracle.sketch_update(oracle.new_counters(p), p, xyz[:12345], g0=0, rate=0.5)
    b = oracle.sketch_update(oracle.new_counters(p), p, xyz[12345:], g0=12345, rate=0.5)
    assert np.array_equal(whole, a + b)                      # sketches sum (Sec. 5)
    par = oracle.sketch_update(oracle.new_counters(p), p, xyz, rate=0.5, nthreads=4)
    assert np.array_equal(whole, par)
    perm = rng.permutation(len(xyz))
    full1 = oracle.sketch_update(oracle.new_counters(p), p, xyz)
    full2 = oracle.sketch_update(oracle.new_counters(p), p, xyz[perm])
    assert np.array_equal(full1, full2)                      # order-free without sampling


def test_counters_wrap_like_int32():
    p = oracle.Params(1, 1, 0.1, 0.1, 0)                      # G = 1, one cell
    C = oracle.new_counters(p)
    b, s = oracle.hash_row(p, 0, (0, 0, 0))
    C[0, b] = np.int32(2**31 - 1) if s > 0 else np.int32(-2**31)
    oracle.sketch_update(C, p, np.zeros((1, 3), np.float32))
    assert C[0, b] == (np.int32(-2**31) if s > 0 else np.int32(2**31 - 1))


# ------------------------------------------------------------ estimate, top-k

def _paper_median(vals):
    """Algorithm 4's rule: a value with at most t/2 estimates above and below."""
    t = len(vals)
    ok = [v for v in vals if sum(u > v for u in vals) <= t / 2 and sum(u < v for u in vals) <= t / 2]
    return ok


def _brute_topk(C, p, k):
    ests = []
    for key in range(p.n_cells):
        c3 = oracle.key_decode(key, p.G)
        rows = []
        for r in range(p.rows):
            s = [int(v) for v in p.seeds[4 * r:4 * r + 4]]
            b, sg = hashref.bucket_sign(c3, s[:3], s[3], p.log2_width)
            rows.append(int(C[r, b]) * sg)
        cands = _paper_median(rows)
        med = sorted(rows)[(p.rows - 1) // 2]
        assert med in cands
        if p.rows % 2:
            assert len(set(cands)) == 1
        ests.append((med, key))
    ests.sort(key=lambda e: (-e[0], e[1]))
    return ests[:k]


@pytest.mark.parametrize("rows", [5, 4, 3, 1])
def test_topk_full_search_equals_brute_force(rows):
    rng = np.random.default_rng(12 + rows)
    p = oracle.Params(rows, 6, 1.6, 0.1, 1000 + rows)        # 4096 cells, 64 buckets
    xyz = _box_points(rng, 4000, 1.6)
    C = oracle.sketch_update(oracle.new_counters(p), p, xyz)
    brute = _brute_topk(C, p, p.n_cells)
    for k in (1, 7, 100, 4096, 5000):
        for nt in (1, 3):
            keys, est = oracle.topk_full(C, p, k, nthreads=nt)
            want = brute[:k]
            assert len(keys) == min(k, p.n_cells)
            assert [int(v) for v in keys] == [w[1] for w in want]
            assert [int(v) for v in est] == [w[0] for w in want]


def test_topk_on_empty_sketch_is_smallest_keys():
    p = oracle.Params(5, 8, 2.0, 0.1, 5)
    C = oracle.new_counters(p)
    keys, est = oracle.topk_full(C, p, 10, nthreads=2)
    assert list(keys) == list(range(10)) and not est.any()


def test_estimator_unbiased_over_seeds():
    # E[h_s(i) * c] = f_i under 2-independent hashing (Sec. 2.2)
    rng = np.random.default_rng(21)
    xyz = _box_points(rng, 3000, 3.2, clusters=3)
    p0 = oracle.Params(1, 4, 3.2, 0.1, 0)
    keys = oracle.keys_of(xyz, p0)
    f = Counter(int(k) for k in keys)
    target, ft = max(f.items(), key=lambda kv: kv[1])
    l2sq = sum(v * v for v in f.values())
    vals = []
    for seed in range(400):
        p = oracle.Params(1, 4, 3.2, 0.1, seed + 1)
        C = oracle.sketch_update(oracle.new_counters(p), p, xyz)
        vals.append(oracle.row_estimates(C, p, target)[0])
    sd = math.sqrt((l2sq - ft * ft) / p0.width)              # per-row standard deviation
    assert abs(np.mean(vals) - ft) < 5 * sd / math.sqrt(len(vals))


# ------------------------------------------------------------- exact counting

def test_exact_counts_and_topk():
    rng = np.random.default_rng(30)
    p = oracle.Params(5, 10, 100.0, 0.1, 1, sample_seed=4)
    xyz = _box_points(rng, 50000, 100.0)
    for rate in (1.0, 0.25):
        keys, cnt = oracle.exact_counts(xyz, p, rate=rate)
        kept = oracle.keep_mask(0, len(xyz), p.sample_seed, rate)
        prod = (xyz[kept] * np.float32(p.inv_cell)).astype(np.float32)
        c = np.mod(np.floor(prod).astype(np.int64), p.G)
        want = Counter((c[:, 0] + p.G * (c[:, 1] + p.G * c[:, 2])).tolist())
        assert dict(zip(keys.tolist(), cnt.tolist())) == dict(want)
        assert np.all(np.diff(keys.astype(np.int64)) > 0)
        tk, tc = oracle.exact_topk(keys, cnt, 50)
        ref = sorted(want.items(), key=lambda kv: (-kv[1], kv[0]))[:50]
        assert list(zip(tk.tolist(), tc.tolist())) == ref
        assert oracle.recall_at_k(tk, keys, cnt, 50) == 1.0
