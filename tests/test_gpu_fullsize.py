"""Parity at the benchmark's full sizes, in the benchmark's launch configuration.

Counters are compared whole (the oracle runs the same stream with private
per-thread counters).  The top-k of the 10^9-particle box is compared entry by
entry with the oracle's exhaustive full search over all 1.25e11 cells, stored
in tests/golden/ by tests/golden/make_fullsize_topk.py (an hour of host cores
per sample rate, so not rerun here); the particles and counters are checked
against that file's digests first.  A top-k over 8e12 cells is out of the
oracle's reach, so that one is checked on samples the oracle computes one by
one: every returned estimate, the ranking, and completeness on sampled mesh
lines (every cell of a sampled line that ranks ahead of the k-th entry must
have been returned), with lines through the returned cells among the samples.
"""
import hashlib
import os
import sys

import numpy as np
import pytest

import oracle
import oracle.learned as OL
import synth

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_fullsize_topk as golden  # noqa: E402

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
def big(hs):
    """The 10^9-particle, 500 Mpc/h box of the benchmark (seed 1), host and device."""
    spec = synth.scale_box(1)
    host = torch.empty((spec.n, 3), dtype=torch.float32).pin_memory()
    synth.HaloBox(spec).generate_into_ptr(host.data_ptr(), 0, spec.n, 0)
    dev = host.cuda()
    yield spec, host.numpy(), dev
    del dev


def ranked(keys, est):
    e = est.astype(np.int64)
    return bool(np.all((e[:-1] > e[1:]) | ((e[:-1] == e[1:]) & (keys[:-1] < keys[1:]))))


def check_complete_on_lines(keys, est, value_of, G, lines):
    """Cells of the given lines (cy + G cz) that rank ahead of the last entry
    must all be among keys; value_of(cells) gives their oracle values."""
    th, last = int(est[-1]), int(keys[-1])
    have = set(keys.tolist())
    cx = np.arange(G, dtype=np.uint64)
    for line in np.unique(np.asarray(lines, np.uint64)):
        cells = cx + np.uint64(G) * line
        v = value_of(cells).astype(np.int64)
        ahead = cells[(v > th) | ((v == th) & (cells < np.uint64(last)))]
        missing = [c for c in ahead.tolist() if c not in have]
        assert not missing, (int(line), missing[:5])


def sample_lines(keys, G, rng, n_random=300, n_from_keys=60):
    kk = np.asarray(keys, np.uint64)
    own = kk[rng.choice(kk.size, min(n_from_keys, kk.size), replace=False)] // np.uint64(G)
    return np.concatenate([rng.integers(0, G * G, n_random).astype(np.uint64), own])


# ---------------------------------------------------------------- 10^9 box

@pytest.mark.parametrize("rate", [1.0, 0.1])
def test_halo_box_1e9_counters_and_topk(hs, big, rate):
    spec, host, dev = big
    meta, gkeys, gest = golden.read_golden(golden.golden_path(rate))
    assert meta["particles_sha256"] == golden.sha256_of(host), "the generator's output differs"
    stream = torch.cuda.current_stream()
    k = 10 ** 4
    sk = hs.Sketch(5, 24, 500.0, 0.1, 1, 2, stream=stream)     # the benchmark's handle
    keys = np.empty(k, np.uint64)
    est = np.empty(k, np.int32)
    hs.sketch_update(sk.h, dev, spec.n, rate)
    hs.sketch_flush(sk.h)
    n = hs.topk_extract(sk.h, k, keys, est)
    counters = sk.counters()
    assert golden.sha256_of(counters) == meta["counters_sha256"]
    p = oracle.Params(5, 24, 500.0, 0.1, 1, 2)
    C = oracle.sketch_update(oracle.new_counters(p), p, host, rate=rate, nthreads=NT)
    assert np.array_equal(counters, C)
    # the whole ranked list equals the oracle's exhaustive search
    assert n == k and gkeys.size == k
    assert np.array_equal(keys, gkeys) and np.array_equal(est, gest)
    assert ranked(keys, est) and len(set(keys.tolist())) == k
    assert np.array_equal(oracle.estimate(C, p, keys), est)
    sk.close()


# ---------------------------------------------------------------- learned, 10^9 box

def centre_router(thr_count):
    P = np.zeros(OL.N_PARAMS, np.float32)
    w1, b1, w2, b2, w3, b3 = OL.unpack(P)
    w1[0, 13] = 1.0
    w2[0, 0] = 1.0
    w3[0] = 1.0
    b3[0] = -OL.bf16_value(OL.feature_of([thr_count]))[0]
    return P


def test_learned_halo_box_1e9(hs, big):
    spec, host, dev = big
    R, tlog2, fseed, frate, k = 10, 20, 64, 1.0 / 64, 10 ** 4
    P = centre_router(24)
    mlp = hs.MLP()
    mlp.set_params(P)
    L = hs.Learned(5, 23, 500.0, 0.1, 1, 2, coarse_factor=R, table_log2=tlog2,
                   feature_seed=fseed, feature_rate=frate)
    L.prepare(dev, mlp, spec.n)
    L.update(dev, spec.n)
    gk, ge = L.topk(k)
    p = oracle.Params(5, 23, 500.0, 0.1, 1, 2)
    Gc = p.G // R
    counts = OL.coarse_hist(host, p, R, fseed, frate)
    assert np.array_equal(L.coarse_counts(), counts)
    okeys = np.flatnonzero(counts).astype(np.uint64)
    ofeat = OL.features(counts, Gc, okeys)
    ologit = OL.forward_f32(P, ofeat, nthreads=NT)
    ck, cl = L.logits()
    o = np.argsort(ck)
    assert np.array_equal(ck[o], okeys)
    assert np.array_equal(cl[o].view(np.uint32), ologit.view(np.uint32))
    B = OL.route_budget(tlog2, R)
    routed = OL.route_bytes(okeys, ologit, Gc, B)
    assert int((ologit > 0).sum()) > B                     # the budget's selection path
    assert np.array_equal(L.routed(), np.flatnonzero(routed).astype(np.uint64))
    C = oracle.new_counters(p)
    tk, tc = OL.learned_update(C, p, host, routed, R, nthreads=NT, cap=B * R ** 3 + 1)
    assert np.array_equal(L.counters(), C)
    lk, lc = L.table()
    assert np.array_equal(lk, tk) and np.array_equal(lc, tc)
    # the merged top-k: exact counts for routed cells, estimates for the rest
    assert len(gk) == k and ranked(gk, ge)
    table = dict(zip(tk.tolist(), tc.tolist()))
    kx = gk.astype(np.int64)
    crd = (kx % p.G) // R + Gc * (((kx // p.G) % p.G) // R + Gc * ((kx // (p.G * p.G)) // R))
    is_routed = routed[crd] == 1
    assert all(ge[i] == table.get(int(gk[i]), 0) for i in np.flatnonzero(is_routed))
    assert np.array_equal(oracle.estimate(C, p, gk[~is_routed]), ge[~is_routed])
    th, last = int(ge[-1]), int(gk[-1])
    have = set(gk.tolist())
    assert all(key in have for key, c in table.items() if c > th or (c == th and key < last))

    def value_of(cells):
        c = cells.astype(np.int64)
        r = routed[(c % p.G) // R + Gc * (((c // p.G) % p.G) // R + Gc * ((c // (p.G * p.G)) // R))]
        v = oracle.estimate(C, p, cells).astype(np.int64)
        v[r == 1] = np.iinfo(np.int64).min                # routed cells: checked through the table
        return v

    check_complete_on_lines(gk, ge, value_of, p.G,
                            sample_lines(gk[~is_routed], p.G, np.random.default_rng(9)))
    L.close()


# ---------------------------------------------------------------- 64 sub-volumes

def test_subvolumes_64_counters_and_topk(hs):
    specs = synth.subvolume_specs(seed=3)
    counts = [s.n for s in specs]
    offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.uint64)
    host = torch.empty((int(offsets[-1]), 3), dtype=torch.float32).pin_memory()
    for s_, o in zip(specs, offsets[:-1]):
        synth.HaloBox(s_).generate_into_ptr(host.data_ptr() + int(o) * 12, 0, s_.n)
    x = host.numpy()
    dev = host.cuda()
    stream = torch.cuda.Stream()
    b = hs.Batch(5, 18, [s_.box for s_ in specs], 0.1, hash_seed=3, sample_seed=4, stream=stream)
    b.autotune(dev, offsets, 1.0)
    b.update(dev, offsets, 1.0)
    res = b.topk(500)
    rng = np.random.default_rng(3)
    for v, s_ in enumerate(specs):
        p = oracle.Params(5, 18, s_.box, 0.1, 3, 4)
        part = x[offsets[v]:offsets[v + 1]]
        C = oracle.sketch_update(oracle.new_counters(p), p, part, nthreads=NT)
        assert np.array_equal(b.counters(v), C), v
        keys, est = res[v]
        if p.n_cells <= 3 * 10 ** 7:
            wk, we = oracle.topk_full(C, p, 500, nthreads=NT)
            assert np.array_equal(keys, wk) and np.array_equal(est, we), v
        else:
            assert len(keys) == 500 and ranked(keys, est), v
            assert np.array_equal(oracle.estimate(C, p, keys), est), v
            check_complete_on_lines(keys, est, lambda c: oracle.estimate(C, p, c), p.G,
                                    sample_lines(keys, p.G, rng, 40, 20))
    b.close()


# ---------------------------------------------------------------- the 8e12-cell stream

def test_stream_geometry_first_chunks(hs):
    """The 2000 Mpc/h stream's first two 1 GB chunks from pinned host memory,
    5 x 2^26 with the 5 x 2^26 super-item layer, rate 0.1, hierarchical top-10^4."""
    spec = synth.stream_box(4)
    C = 10 ** 9 // 12
    hb = synth.HaloBox(spec)
    chunks = [torch.empty((C, 3), dtype=torch.float32).pin_memory() for _ in range(2)]
    for c, buf in enumerate(chunks):
        hb.generate_into_ptr(buf.data_ptr(), c * C, C)
    F, cm, k, rate = 10, 2, 10 ** 4, 0.1
    sk = hs.Sketch(5, 26, 2000.0, 0.1, 5, 6)
    sk.set_hierarchy(F, 26, cm)
    for buf in chunks:
        sk.update(buf, rate=rate)
    hs.sketch_wait_copies(sk.h)
    keys, est = sk.topk(k)
    x = np.concatenate([buf.numpy() for buf in chunks])
    p = oracle.Params(5, 26, 2000.0, 0.1, 5, 6)
    q = oracle.super_params(p, F, 26)
    C2 = oracle.sketch_update(oracle.new_counters(p), p, x, rate=rate, nthreads=NT)
    assert np.array_equal(sk.counters(), C2)
    C1 = oracle.sketch_update_super(oracle.new_counters(q), p, q, F, x, rate=rate)
    assert np.array_equal(sk.super_counters(), C1)
    # first layer: the c*k best super-items (the super sketch's own top-k)
    ms = cm * k
    skeys = np.empty(ms, np.uint64)
    sest = np.empty(ms, np.int32)
    assert hs.topk_extract(sk.super_handle(), ms, skeys, sest) == ms
    assert ranked(skeys, sest)
    assert np.array_equal(oracle.estimate(C1, q, skeys), sest)
    rng = np.random.default_rng(4)
    check_complete_on_lines(skeys, sest, lambda c: oracle.estimate(C1, q, c), q.G,
                            sample_lines(skeys, q.G, rng, 200, 40))
    # second layer: the k best cells of those super-items
    assert len(keys) == k and ranked(keys, est)
    assert np.array_equal(oracle.estimate(C2, p, keys), est)
    kx = keys.astype(np.int64)
    sup = (kx % p.G) // F + q.G * (((kx // p.G) % p.G) // F + q.G * ((kx // (p.G * p.G)) // F))
    sset = set(skeys.tolist())
    assert all(int(s) in sset for s in sup)
    th, last = int(est[-1]), int(keys[-1])
    have = set(keys.tolist())
    l = np.arange(F ** 3)
    for s in rng.choice(skeys, 150, replace=False).astype(np.int64):
        sx, sy, sz = s % q.G, (s // q.G) % q.G, s // (q.G * q.G)
        cells = ((sx * F + l % F) + p.G * ((sy * F + (l // F) % F) + p.G * (sz * F + l // (F * F))))
        cells = cells.astype(np.uint64)
        v = oracle.estimate(C2, p, cells).astype(np.int64)
        ahead = cells[(v > th) | ((v == th) & (cells < np.uint64(last)))]
        assert all(c in have for c in ahead.tolist()), int(s)
    sk.close()
