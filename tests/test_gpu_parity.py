"""GPU path vs the CPU oracle, through the C ABI: counters, estimates and top-k
must match bit for bit (integer work; the only float op, the quantisation
multiply, is one float32 rounding on both sides)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

NT = oracle.default_threads()


@pytest.fixture(scope="module")
def hs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_00975_gb300 import halosketch
    halosketch.lib()
    return halosketch


@pytest.fixture(scope="module")
def small():
    spec = synth.small_box(0)
    return spec, synth.HaloBox(spec).generate()


# "inline": the directory with every slot's first records inline (the layout
# large meshes use), forced on the small meshes the oracle searches in full
SEARCH = {"auto": 0, "scan": 1, "directory": 2, "inline": 2 | 16}
UPDATE = {"auto": 0, "direct": 4, "binned": 8}


def _pair(hs, rows, log2w, box, cell, hash_seed, sample_seed=0, flags=0):
    sk = hs.Sketch(rows, log2w, box, cell, hash_seed, sample_seed, flags=flags)
    p = oracle.Params(rows, log2w, box, cell, hash_seed, sample_seed)
    return sk, p


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


# ---------------------------------------------------------------- update mode

@pytest.mark.parametrize("rate", [1.0, 0.1, 1.0 / 16])
@pytest.mark.parametrize("update", list(UPDATE))
def test_update_small_box_bitexact(hs, small, rate, update):
    spec, xyz = small
    sk, p = _pair(hs, 5, 16, spec.box, 0.1, 11, 22, flags=UPDATE[update])
    sk.update(_dev(xyz), rate=rate)
    want = oracle.sketch_update(oracle.new_counters(p), p, xyz, rate=rate, nthreads=NT)
    assert np.array_equal(sk.counters(), want)
    assert sk.info().n_seen == len(xyz)


@pytest.mark.parametrize("update", list(UPDATE))
def test_update_ragged_calls_and_alignment(hs, small, update):
    # uneven call sizes keep the global particle index running across calls;
    # the 1-particle offsets give 12-byte (unaligned) starts
    spec, xyz = small
    sk, p = _pair(hs, 5, 12, spec.box, 0.1, 5, 9, flags=UPDATE[update])
    d = _dev(xyz)
    sizes = [0, 1, 3, 4, 5, 1023, 100003, 7, 64, 250001]
    off = 0
    want = oracle.new_counters(p)
    for n in sizes:
        sk.update(d[off:off + n], n, rate=0.5)
        oracle.sketch_update(want, p, xyz[off:off + n], g0=off, rate=0.5, nthreads=NT)
        off += n
    assert np.array_equal(sk.counters(), want)


def test_update_from_host_buffers(hs, small):
    spec, xyz = small
    sk, p = _pair(hs, 5, 16, spec.box, 0.1, 3, 4)
    pinned = torch.from_numpy(xyz[:600000]).pin_memory()
    sk.update(xyz[600000:700001])                 # pageable numpy
    sk.update(pinned)                             # pinned torch
    want = oracle.new_counters(p)
    oracle.sketch_update(want, p, xyz[600000:700001], g0=0, nthreads=NT)
    oracle.sketch_update(want, p, xyz[:600000], g0=100001, nthreads=NT)
    assert np.array_equal(sk.counters(), want)


@pytest.mark.parametrize("rows,log2w", [(1, 10), (3, 14), (4, 8), (7, 18), (32, 6), (5, 24),
                                       (7, 24), (5, 26)])
@pytest.mark.parametrize("update", ["direct", "binned"])
def test_update_other_shapes(hs, small, rows, log2w, update):
    spec, xyz = small
    sk, p = _pair(hs, rows, log2w, spec.box, 0.1, 100 + rows, 1, flags=UPDATE[update])
    sk.update(_dev(xyz[:300000]), rate=0.7)
    want = oracle.sketch_update(oracle.new_counters(p), p, xyz[:300000], rate=0.7, nthreads=NT)
    assert np.array_equal(sk.counters(), want)


@pytest.mark.parametrize("update", ["direct", "binned"])
def test_update_edge_coordinates(hs, update):
    sk, p = _pair(hs, 5, 10, 100.0, 0.1, 1, flags=UPDATE[update])
    pts = np.array([[0, 0, 0], [100.0, 99.99999, -0.05], [0.7, 0.3, 250.0], [-1e-30, 5e9, 1],
                    [np.nan, 1, 1], [1, np.inf, 2], [3e9, -3e9, 1], [1, 2, 3]], np.float32)
    pts = np.repeat(pts, 3, axis=0)
    sk.update(_dev(pts))
    want = oracle.sketch_update(oracle.new_counters(p), p, pts)
    assert np.array_equal(sk.counters(), want)


@pytest.mark.parametrize("update", ["direct", "binned"])
def test_counter_wraparound(hs, update):
    sk, p = _pair(hs, 3, 4, 0.1, 0.1, 0, flags=UPDATE[update])    # one cell
    c = np.zeros((3, 16), np.int32)
    for r in range(3):
        b, s = oracle.hash_row(p, r, (0, 0, 0))
        c[r, b] = 2**31 - 1 if s > 0 else -2**31
    sk.load_counters(c)
    sk.update(_dev(np.zeros((2, 3), np.float32)))
    want = c.copy()
    oracle.sketch_update(want, p, np.zeros((2, 3), np.float32))
    assert np.array_equal(sk.counters(), want)


def test_merge_is_the_sketch_of_the_union(hs, small):
    spec, xyz = small
    a, p = _pair(hs, 5, 14, spec.box, 0.1, 8, 8)
    b, _ = _pair(hs, 5, 14, spec.box, 0.1, 8, 8)
    a.update(_dev(xyz[:400000]))
    b.update(_dev(xyz[400000:]))
    a.merge(b)
    want = oracle.sketch_update(oracle.new_counters(p), p, xyz, nthreads=NT)
    assert np.array_equal(a.counters(), want)
    c, _ = _pair(hs, 5, 13, spec.box, 0.1, 8, 8)
    with pytest.raises(hs.HSError):
        a.merge(c)


def test_binned_skew_overflows_to_direct_adds(hs):
    # every particle in a handful of cells: the shared-memory buffers of those
    # bins overflow on every tile and the excess goes through global atomics
    rng = np.random.default_rng(3)
    sk, p = _pair(hs, 5, 20, 100.0, 0.1, 12, flags=UPDATE["binned"])
    cells = np.array([[10.05, 20.05, 30.05], [70.05, 5.05, 99.95], [0.05, 0.05, 0.05]], np.float32)
    pts = np.concatenate([cells[rng.integers(0, 3, 3_000_000)],
                          rng.uniform(0, 100, (200_000, 3)).astype(np.float32)])
    sk.update(_dev(pts), rate=0.9)
    want = oracle.sketch_update(oracle.new_counters(p), p, pts, rate=0.9, nthreads=NT)
    assert np.array_equal(sk.counters(), want)


def test_binned_pending_across_calls_and_readers(hs, small):
    # increments stay in the bins across calls; every reader drains them first
    spec, xyz = small
    sk, p = _pair(hs, 5, 16, spec.box, 0.1, 77, 5, flags=UPDATE["binned"])
    want = oracle.new_counters(p)
    d = _dev(xyz)
    sk.update(d[:300000], 300000, rate=0.5)
    oracle.sketch_update(want, p, xyz[:300000], g0=0, rate=0.5, nthreads=NT)
    keys = oracle.keys_of(xyz[:1000], p)
    assert np.array_equal(sk.query(keys), oracle.estimate(want, p, keys))
    sk.update(d[300000:], len(xyz) - 300000, rate=0.5)
    oracle.sketch_update(want, p, xyz[300000:], g0=300000, rate=0.5, nthreads=NT)
    k1, e1 = sk.topk(500)
    wk, we = oracle.topk_full(want, p, 500, nthreads=NT)
    assert np.array_equal(k1, wk) and np.array_equal(e1, we)
    sk.update(d[:1000], 1000)
    sk.reset()                                   # pending codes are dropped, not applied
    assert not sk.counters().any()


def test_shards_with_seek_merge_to_the_whole_stream(hs, small):
    # each shard keeps its global indices (sampling unchanged) and its own probe
    spec, xyz = small
    whole, p = _pair(hs, 5, 16, spec.box, 0.1, 44, 6)
    a, _ = _pair(hs, 5, 16, spec.box, 0.1, 44, 6)
    b, _ = _pair(hs, 5, 16, spec.box, 0.1, 44, 6)
    whole.update(_dev(xyz), rate=0.3)
    cut = 654321
    a.update(_dev(xyz[:cut]), rate=0.3)
    b.seek(cut)
    b.update(_dev(xyz[cut:]), rate=0.3)
    kb, eb = b.topk(100)                        # uses b's own probe (no global index < 2^20)
    Cb = oracle.sketch_update(oracle.new_counters(p), p, xyz[cut:], g0=cut, rate=0.3, nthreads=NT)
    assert np.array_equal(b.counters(), Cb)
    wk, we = oracle.topk_full(Cb, p, 100, nthreads=NT)
    assert np.array_equal(kb, wk) and np.array_equal(eb, we)
    a.merge(b)
    assert np.array_equal(a.counters(), whole.counters())
    k1, e1 = a.topk(300)
    k2, e2 = whole.topk(300)
    assert np.array_equal(k1, k2) and np.array_equal(e1, e2)


def test_reset(hs, small):
    spec, xyz = small
    sk, p = _pair(hs, 5, 12, spec.box, 0.1, 2)
    sk.update(_dev(xyz[:1000]))
    sk.reset()
    assert not sk.counters().any() and sk.info().n_seen == 0


# --------------------------------------------------------------- estimate mode

def test_point_query(hs, small):
    spec, xyz = small
    sk, p = _pair(hs, 5, 16, spec.box, 0.1, 7)
    sk.update(_dev(xyz))
    C = oracle.sketch_update(oracle.new_counters(p), p, xyz, nthreads=NT)
    rng = np.random.default_rng(0)
    keys = np.concatenate([oracle.keys_of(xyz[:5000], p),
                           rng.integers(0, p.n_cells, 5000, dtype=np.uint64)])
    assert np.array_equal(sk.query(keys), oracle.estimate(C, p, keys))
    dkeys, dest = _dev(keys), torch.empty(keys.size, dtype=torch.int32, device="cuda")
    hs.sketch_query(sk.h, dkeys, dest)
    assert np.array_equal(dest.cpu().numpy(), oracle.estimate(C, p, keys))
    with pytest.raises(hs.HSError):
        sk.query(np.array([p.n_cells], np.uint64))


@pytest.mark.parametrize("search", list(SEARCH))
def test_topk_small_box_bitexact(hs, small, search):
    spec, xyz = small
    sk, p = _pair(hs, 5, 16, spec.box, 0.1, 13, flags=SEARCH[search])
    sk.update(_dev(xyz))
    C = oracle.sketch_update(oracle.new_counters(p), p, xyz, nthreads=NT)
    assert np.array_equal(sk.counters(), C)
    keys, est = sk.topk(1000)
    wk, we = oracle.topk_full(C, p, 1000, nthreads=NT)
    assert np.array_equal(keys, wk) and np.array_equal(est, we)


@pytest.mark.parametrize("rows,log2w,G,k", [(5, 6, 16, 50), (5, 8, 40, 4000), (3, 7, 24, 300),
                                            (4, 5, 20, 100), (1, 9, 30, 77), (7, 10, 36, 500),
                                            (5, 4, 12, 1728), (5, 4, 12, 5000)])
@pytest.mark.parametrize("search", list(SEARCH))
def test_topk_small_dictionaries_bitexact(hs, rows, log2w, G, k, search):
    # narrow sketches: many collisions, ties and negative estimates
    rng = np.random.default_rng(rows * 1000 + G)
    box = G * 0.1
    sk, p = _pair(hs, rows, log2w, box, 0.1, 50 + G, flags=SEARCH[search])
    centres = rng.uniform(0, box, (6, 3))
    pts = centres[rng.integers(0, 6, 20000)] + rng.normal(0, box / 20, (20000, 3))
    pts = np.mod(pts, box).astype(np.float32)
    sk.update(_dev(pts))
    C = oracle.sketch_update(oracle.new_counters(p), p, pts, nthreads=NT)
    assert np.array_equal(sk.counters(), C)
    keys, est = sk.topk(k)
    wk, we = oracle.topk_full(C, p, k, nthreads=NT)
    assert len(keys) == min(k, G ** 3)
    assert np.array_equal(keys, wk) and np.array_equal(est, we)


@pytest.mark.parametrize("search", list(SEARCH))
def test_topk_loaded_random_counters(hs, search):
    # arbitrary counters (any sign, any magnitude) through the same search
    rng = np.random.default_rng(77)
    for rows, log2w, G, k in [(5, 10, 50, 2000), (5, 12, 64, 3000), (6, 9, 33, 1000)]:
        sk, p = _pair(hs, rows, log2w, G * 0.1, 0.1, rows + G, flags=SEARCH[search])
        C = rng.integers(-50, 50, size=(rows, 1 << log2w)).astype(np.int32)
        C[:, ::97] = rng.integers(-2**31, 2**31 - 1, size=C[:, ::97].shape)
        sk.load_counters(C)
        keys, est = sk.topk(k)
        wk, we = oracle.topk_full(C, p, k, nthreads=NT)
        assert np.array_equal(keys, wk) and np.array_equal(est, we)


def test_topk_empty_sketch_ties(hs):
    # every estimate is 0: the k smallest keys, through the tie path
    sk, p = _pair(hs, 5, 16, 100.0, 0.1, 1)
    keys, est = sk.topk(1000)
    assert np.array_equal(keys, np.arange(1000, dtype=np.uint64)) and not est.any()


def test_topk_single_heavy_cell_many_ties(hs):
    # one occupied cell: it ranks first with its exact count; every other cell
    # estimates 0 (it could only differ by colliding with the heavy cell in 3 of
    # 5 rows, about 1e9 * 10 * 2^-60 expected cells), so the rest are the
    # smallest keys - reached through the tie path
    sk, p = _pair(hs, 5, 20, 100.0, 0.1, 4)
    pts = np.tile(np.array([[50.05, 50.05, 50.05]], np.float32), (333, 1))
    sk.update(_dev(pts))
    keys, est = sk.topk(64)
    heavy = int(oracle.keys_of(pts[:1], p)[0])
    assert [int(v) for v in keys] == [heavy] + list(range(63))
    assert [int(v) for v in est] == [333] + [0] * 63
    C = oracle.sketch_update(oracle.new_counters(p), p, pts)
    assert np.array_equal(oracle.estimate(C, p, keys), est)


@pytest.mark.parametrize("search", list(SEARCH))
def test_topk_after_reset_and_requery(hs, small, search):
    spec, xyz = small
    sk, p = _pair(hs, 5, 16, spec.box, 0.1, 21, flags=SEARCH[search])
    sk.update(_dev(xyz[:500000]))
    k1 = sk.topk(200)
    k1b = sk.topk(200)
    assert np.array_equal(k1[0], k1b[0]) and np.array_equal(k1[1], k1b[1])
    sk.reset()
    sk.update(_dev(xyz[500000:]))
    C = oracle.sketch_update(oracle.new_counters(p), p, xyz[500000:], nthreads=NT)
    assert np.array_equal(sk.counters(), C)
    keys, est = sk.topk(300)
    wk, we = oracle.topk_full(C, p, 300, nthreads=NT)
    assert np.array_equal(keys, wk) and np.array_equal(est, we)


@pytest.mark.parametrize("search", ["scan", "directory", "inline"])
def test_topk_heavy_ties_at_positive_threshold(hs, search):
    # many cells share the k-th estimate (every occupied cell has count 3):
    # the positive-threshold tie path must return the smallest keys among them
    rng = np.random.default_rng(5)
    sk, p = _pair(hs, 5, 20, 30.0, 0.1, 9, flags=SEARCH[search])
    cells = rng.choice(300 ** 3, size=4000, replace=False)
    cx, cy, cz = cells % 300, (cells // 300) % 300, cells // 90000
    pts = (np.stack([cx, cy, cz], 1).astype(np.float64) * 0.1 + 0.05).astype(np.float32)
    pts = np.repeat(pts, 3, axis=0)
    sk.update(_dev(pts))
    C = oracle.sketch_update(oracle.new_counters(p), p, pts, nthreads=NT)
    assert np.array_equal(sk.counters(), C)
    keys, est = sk.topk(1500)
    wk, we = oracle.topk_full(C, p, 1500, nthreads=NT)
    assert np.array_equal(keys, wk) and np.array_equal(est, we)


@pytest.mark.parametrize("search", list(SEARCH))
def test_topk_overflow_tie_path_positive_threshold(hs, search):
    # all counters 1: every estimate is +1 or -1 and about 8.4e6 of the 2^24
    # cells tie at +1, more than the candidate buffer holds - the search must
    # raise its threshold, fail to separate the ties, and take them in key order
    sk, p = _pair(hs, 5, 16, 25.6, 0.1, 31, flags=SEARCH[search])
    C = np.ones((5, 1 << 16), np.int32)
    sk.load_counters(C)
    keys, est = sk.topk(2000)
    wk, we = oracle.topk_full(C, p, 2000, nthreads=NT)
    assert np.array_equal(keys, wk) and np.array_equal(est, we)
    assert (we == 1).all()
    st = sk.stats()
    assert st["last_passes"] >= 3
