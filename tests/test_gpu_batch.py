"""Batches of independent sub-volumes through the C ABI: every volume's
counters and top-k must equal a separate oracle sketch of that volume."""
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


def _volumes(counts, seed):
    """Uneven sub-volumes with the small-box mixture scaled to each size."""
    specs, parts = [], []
    for i, n in enumerate(counts):
        L = max(0.5, round(8.0 * (n / 20000) ** (1 / 3) / 0.1) * 0.1)
        spec = synth.BoxSpec(n=n, box=L, n_halo=max(1, n // 1000), seed=seed * 100 + i)
        specs.append(spec)
        parts.append(synth.HaloBox(spec).generate() if n else np.zeros((0, 3), np.float32))
    offsets = np.concatenate([[0], np.cumsum([p.shape[0] for p in parts])]).astype(np.uint64)
    return specs, np.concatenate(parts), offsets


def _oracle_counters(spec, xyz, p, g0=0, rate=1.0, C=None):
    C = oracle.new_counters(p) if C is None else C
    return oracle.sketch_update(C, p, xyz, g0=g0, rate=rate, nthreads=NT)


@pytest.mark.parametrize("rate", [1.0, 0.3])
def test_batch_counters_and_topk_equal_separate_sketches(hs, rate):
    counts = [20000, 3, 150000, 0, 77777, 400001]
    specs, xyz, off = _volumes(counts, 1)
    b = hs.Batch(5, 14, [s.box for s in specs], 0.1, hash_seed=5, sample_seed=6)
    d = torch.from_numpy(xyz).cuda()
    b.update(d, off, rate)
    b.update(d, off, rate)                       # replayed graph, indices continue
    res = b.topk(300)
    for v, spec in enumerate(specs):
        p = oracle.Params(5, 14, spec.box, 0.1, 5, 6)
        part = xyz[off[v]:off[v + 1]]
        C = _oracle_counters(spec, part, p, 0, rate)
        C = _oracle_counters(spec, part, p, len(part), rate, C)
        assert np.array_equal(b.counters(v), C), v
        assert b.info(v).n_seen == 2 * len(part)
        wk, we = oracle.topk_full(C, p, 300, nthreads=NT)
        assert np.array_equal(res[v][0], wk) and np.array_equal(res[v][1], we), v
    # the empty and the 3-particle volume have fewer probe cells than k: the
    # per-volume path answers them
    assert 2 <= b.stats()["host_path_volumes"] < len(counts)
    b.close()


@pytest.mark.parametrize("search", [1, 2])
def test_batch_topk_both_search_methods(hs, search):
    counts = [60000, 90000, 30000]
    specs, xyz, off = _volumes(counts, 2)
    b = hs.Batch(5, 12, [s.box for s in specs], 0.1, hash_seed=7, sample_seed=1, flags=search)
    b.update(torch.from_numpy(xyz).cuda(), off)
    res = b.topk(500)
    st = b.stats()
    if search == 1:          # a scan is asked for: every volume by the per-volume path
        assert st["host_path_volumes"] == len(counts)
    for v, spec in enumerate(specs):
        p = oracle.Params(5, 12, spec.box, 0.1, 7, 1)
        C = _oracle_counters(spec, xyz[off[v]:off[v + 1]], p)
        wk, we = oracle.topk_full(C, p, 500, nthreads=NT)
        assert np.array_equal(res[v][0], wk) and np.array_equal(res[v][1], we)
    b.close()


def test_batch_autotune_then_exact(hs):
    counts = [250000, 120000, 333333, 50000]
    specs, xyz, off = _volumes(counts, 3)
    b = hs.Batch(5, 16, [s.box for s in specs], 0.1, hash_seed=11, sample_seed=2)
    d = torch.from_numpy(xyz).cuda()
    tune = b.autotune(d, off, 0.5)
    assert tune["configs_tried"] >= 2 and tune["rounds"] == 1
    assert b.info(0).n_seen == 0 and not b.counters(1).any()     # tuning reset the batch
    b.update(d, off, 0.5)
    for v, spec in enumerate(specs):
        p = oracle.Params(5, 16, spec.box, 0.1, 11, 2)
        C = _oracle_counters(spec, xyz[off[v]:off[v + 1]], p, rate=0.5)
        assert np.array_equal(b.counters(v), C)
    b.reset()
    assert not b.counters(2).any()
    # a second batch of the same shape takes the kept choice without running
    b2 = hs.Batch(5, 16, [s.box for s in specs], 0.1, hash_seed=11, sample_seed=2)
    tune2 = b2.autotune(d, off, 0.5)
    assert tune2["configs_tried"] == 0 and tune2["slot"] == tune["slot"]
    assert tune2["window_volumes"] == tune["window_volumes"] in (1, 2, 4)
    b2.update(d, off, 0.5)
    for v, spec in enumerate(specs):
        p = oracle.Params(5, 16, spec.box, 0.1, 11, 2)
        C = _oracle_counters(spec, xyz[off[v]:off[v + 1]], p, rate=0.5)
        assert np.array_equal(b2.counters(v), C)
    b2.close()
    b.close()


@pytest.mark.parametrize("rate", [1.0, 0.1])
def test_batch_many_tiny_volumes(hs, rate):
    """Scatter tiles (3072 particles) that span more volumes than the ring
    window holds: those cells are added directly, and the sums still equal
    separate sketches.  Empty volumes sit between the tiny ones."""
    rng = np.random.default_rng(5)
    counts = [int(c) for c in rng.integers(1, 1500, size=40)]
    counts[3] = counts[17] = counts[18] = 0
    counts += [200000, 5, 90000]
    specs, xyz, off = _volumes(counts, 4)
    b = hs.Batch(5, 15, [s.box for s in specs], 0.1, hash_seed=13, sample_seed=14)
    b.update(torch.from_numpy(xyz).cuda(), off, rate)
    for v, spec in enumerate(specs):
        p = oracle.Params(5, 15, spec.box, 0.1, 13, 14)
        C = _oracle_counters(spec, xyz[off[v]:off[v + 1]], p, rate=rate)
        assert np.array_equal(b.counters(v), C), v
    b.close()


@pytest.mark.parametrize("rate", [1.0, 0.1])
def test_batch_sub_volume_sketch_size(hs, rate):
    """5 x 2^18 sketches (eight 2^15-counter bins a row): the ring window
    then holds whole volumes' bins, and volume boundaries fall inside tiles."""
    counts = [700001, 65536, 1234567, 3071, 500000]
    specs, xyz, off = _volumes(counts, 5)
    b = hs.Batch(5, 18, [s.box for s in specs], 0.1, hash_seed=15, sample_seed=16)
    d = torch.from_numpy(xyz).cuda()
    b.update(d, off, rate)
    b.update(d, off, rate)
    res = b.topk(500)
    for v, spec in enumerate(specs):
        p = oracle.Params(5, 18, spec.box, 0.1, 15, 16)
        part = xyz[off[v]:off[v + 1]]
        C = _oracle_counters(spec, part, p, 0, rate)
        C = _oracle_counters(spec, part, p, len(part), rate, C)
        assert np.array_equal(b.counters(v), C), v
        wk, we = oracle.topk_full(C, p, 500, nthreads=NT)
        assert np.array_equal(res[v][0], wk) and np.array_equal(res[v][1], we), v
    b.close()


@pytest.mark.parametrize("k,log2w", [(1, 16), (64, 16), (1000, 16), (300, 14)])
def test_batch_device_topk_every_volume(hs, k, log2w):
    """Volumes whose probes hold enough cells: the single-graph query answers
    all of them (no per-volume path), repeatedly and after more updates, and
    equals the oracle's exhaustive search.  With W = 2^14 < G^2 each
    directory has more slots than buckets and a bucket's lines span a run of
    slots."""
    counts = [300000, 450000, 260000, 600000]
    specs, xyz, off = _volumes(counts, 6)
    b = hs.Batch(5, log2w, [s.box for s in specs], 0.1, hash_seed=17, sample_seed=18)
    d = torch.from_numpy(xyz).cuda()
    Cs = [None] * len(specs)
    for rnd in range(2):
        b.update(d, off, 1.0)
        res = b.topk(k)
        assert b.stats()["host_path_volumes"] == 0
        for v, spec in enumerate(specs):
            p = oracle.Params(5, log2w, spec.box, 0.1, 17, 18)
            part = xyz[off[v]:off[v + 1]]
            Cs[v] = _oracle_counters(spec, part, p, rnd * len(part), 1.0, Cs[v])
            wk, we = oracle.topk_full(Cs[v], p, k, nthreads=NT)
            assert np.array_equal(res[v][0], wk) and np.array_equal(res[v][1], we), (rnd, v)
    b.close()


def test_batch_argument_errors(hs):
    with pytest.raises(hs.HSError):
        hs.Batch(5, 14, [], 0.1)
    b = hs.Batch(5, 14, [10.0, 20.0], 0.1)
    x = torch.zeros((10, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(hs.HSError):
        b.update(x, np.array([0, 6, 4], np.uint64))         # decreasing offsets
    with pytest.raises(hs.HSError):
        b.update(x.cpu().numpy(), np.array([0, 5, 10], np.uint64))   # host particles
    b.close()
