"""Host buffers, against the CPU oracle.

An update from pageable host memory copies the buffer to the device in pieces
of 2^24 particles and runs one binned scatter launch per piece (Add of
Sec. 2.2 per particle, Algorithm 1's stream processing); every launch
continues the same per-block code regions.  Page-locked host memory is read by
the scatter over the host link directly.  Here the stream spans five full
pieces and a ragged sixth, from both kinds of memory, at sample rates 1 and
0.1; the counters and the full-search top-k (Algorithm 1's query, the CSFS
design of Sec. 3.1) must equal the oracle's bit for bit.  The learned
router's sample and update passes stage host buffers in pieces too (three
pieces and a tail).
"""
import numpy as np
import pytest

import oracle
import oracle.learned as OL
import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

NT = oracle.default_threads()
PIECE = 1 << 24


@pytest.fixture(scope="module")
def hs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_00975_gb300 import halosketch
    halosketch.lib()
    return halosketch


@pytest.fixture(scope="module")
def box():
    """5 pieces and a ragged tail in a 100 Mpc/h box (10^9 cells of 0.1 Mpc/h)."""
    n = 5 * PIECE + 12345
    spec = synth.BoxSpec(n=n, box=100.0, n_halo=80000, seed=21)
    xyz = synth.HaloBox(spec).generate()
    return spec, xyz


@pytest.mark.parametrize("rate", [1.0, 0.1])
@pytest.mark.parametrize("memory", ["pinned", "pageable"])
def test_binned_update_from_host_memory(hs, box, rate, memory):
    spec, xyz = box
    src = torch.from_numpy(xyz).pin_memory() if memory == "pinned" else xyz
    sk = hs.Sketch(5, 24, spec.box, 0.1, hash_seed=31, sample_seed=32)
    sk.update(src, rate=rate)
    keys, est = sk.topk(1000)
    st = sk.stats()
    # binned; staged pageable memory takes one launch a piece
    assert st["update_launches"] >= (6 if memory == "pageable" else 1) and st["flush_launches"] >= 1
    assert st["h2d_bytes"] == 12 * spec.n
    p = oracle.Params(5, 24, spec.box, 0.1, 31, 32)
    C = oracle.sketch_update(oracle.new_counters(p), p, xyz, rate=rate, nthreads=NT)
    assert np.array_equal(sk.counters(), C)
    wk, we = oracle.topk_full(C, p, 1000, nthreads=NT)
    assert np.array_equal(keys, wk) and np.array_equal(est, we)
    sk.close()


def test_host_pieces_continue_one_stream(hs, box):
    """Two host calls whose pieces straddle: the particle index (and so the
    sampling) runs on across calls."""
    spec, xyz = box
    cut = 2 * PIECE + 777
    sk = hs.Sketch(5, 24, spec.box, 0.1, hash_seed=5, sample_seed=6)
    sk.update(xyz[:cut], rate=0.5)
    sk.update(torch.from_numpy(xyz[cut:]).pin_memory(), rate=0.5)
    p = oracle.Params(5, 24, spec.box, 0.1, 5, 6)
    C = oracle.sketch_update(oracle.new_counters(p), p, xyz, rate=0.5, nthreads=NT)
    assert np.array_equal(sk.counters(), C)
    sk.close()


def centre_router(thr_count):
    """A router that routes a coarse cell iff its own sample count reaches thr_count."""
    P = np.zeros(OL.N_PARAMS, np.float32)
    w1, b1, w2, b2, w3, b3 = OL.unpack(P)
    w1[0, 13] = 1.0
    w2[0, 0] = 1.0
    w3[0] = 1.0
    b3[0] = -OL.bf16_value(OL.feature_of([thr_count]))[0]
    return P


def test_learned_sample_and_update_from_host_pieces(hs, box):
    spec, xyz = box
    n = 3 * PIECE + 4321
    part = xyz[:n]
    R, tlog2, fseed, frate = 10, 14, 64, 1.0 / 8
    P = centre_router(3)
    mlp = hs.MLP()
    mlp.set_params(P)
    L = hs.Learned(5, 22, spec.box, 0.1, 9, 10, coarse_factor=R, table_log2=tlog2,
                   feature_seed=fseed, feature_rate=frate)
    L.prepare(torch.from_numpy(part).pin_memory(), mlp, n)      # sample pass from host pieces
    L.update(part, n, 0.5)                                       # update pass from pageable pieces
    p = oracle.Params(5, 22, spec.box, 0.1, 9, 10)
    Gc = p.G // R
    counts = OL.coarse_hist(part, p, R, fseed, frate)
    assert np.array_equal(L.coarse_counts(), counts)
    okeys = np.flatnonzero(counts).astype(np.uint64)
    ologit = OL.forward_f32(P, OL.features(counts, Gc, okeys), nthreads=NT)
    B = OL.route_budget(tlog2, R)
    routed = OL.route_bytes(okeys, ologit, Gc, B)
    assert routed.sum() > 0
    assert np.array_equal(L.routed(), np.flatnonzero(routed).astype(np.uint64))
    C = oracle.new_counters(p)
    tk, tc = OL.learned_update(C, p, part, routed, R, rate=0.5, nthreads=NT, cap=B * R ** 3 + 1)
    assert np.array_equal(L.counters(), C)
    lk, lc = L.table()
    assert np.array_equal(lk, tk) and np.array_equal(lc, tc)
    L.close()
    mlp.close()
