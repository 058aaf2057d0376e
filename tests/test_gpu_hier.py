"""Hierarchical query (Algorithm 3, CSHi) on the GPU vs the CPU oracle.

Both layers' counters and the ranked top-k must match bit for bit; with c*k
covering every super-item the hierarchy must give the flat full search."""
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


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.fixture(scope="module")
def data():
    return synth.HaloBox(synth.BoxSpec(n=1 << 18, box=25.6, n_halo=250, seed=21)).generate()


def pair(hs, F, rows=5, log2w=14, slog2w=12, c_mult=2, hash_seed=3, sample_seed=4):
    sk = hs.Sketch(rows, log2w, 25.6, 0.1, hash_seed, sample_seed)
    sk.set_hierarchy(F, slog2w, c_mult)
    p = oracle.Params(rows, log2w, 25.6, 0.1, hash_seed, sample_seed)
    q = oracle.super_params(p, F, slog2w)
    return sk, p, q


@pytest.mark.parametrize("F,rate,host", [(8, 1.0, False), (4, 0.5, False), (8, 0.25, True)])
def test_both_layers_bitexact(hs, data, F, rate, host):
    sk, p, q = pair(hs, F)
    x = data
    src = x if host else _dev(x)
    cut = len(x) // 3 + 7
    sk.update(src[:cut], rate=rate)
    sk.update(src[cut:], rate=rate)
    C2 = oracle.sketch_update(oracle.new_counters(p), p, x, rate=rate, nthreads=NT)
    C1 = oracle.sketch_update_super(oracle.new_counters(q), p, q, F, x, rate=rate)
    assert np.array_equal(sk.counters(), C2)
    assert np.array_equal(sk.super_counters(), C1)


@pytest.mark.parametrize("F,c_mult", [(8, 2), (4, 3)])
def test_hier_topk_bitexact(hs, data, F, c_mult):
    sk, p, q = pair(hs, F, c_mult=c_mult)
    sk.update(_dev(data))
    C2 = oracle.sketch_update(oracle.new_counters(p), p, data, nthreads=NT)
    C1 = oracle.sketch_update_super(oracle.new_counters(q), p, q, F, data)
    wk, we = oracle.topk_hier(C2, p, C1, q, F, 500, c_mult, nthreads=NT)
    for k in (1, 50, 500):
        gk, ge = sk.topk(k)
        vk, ve = oracle.topk_hier(C2, p, C1, q, F, k, c_mult, nthreads=NT) if k != 500 else (wk, we)
        assert np.array_equal(gk, vk) and np.array_equal(ge, ve), k


def test_hier_ties_across_key_windows(hs):
    # few particles and a large k: most of the c*k*F^3 = 5.2e6 candidates tie at
    # estimate 0, more than the candidate buffer holds at once
    x = synth.HaloBox(synth.BoxSpec(n=3000, box=25.6, n_halo=5, seed=5)).generate()
    F, k, cm = 8, 5000, 2
    sk, p, q = pair(hs, F, log2w=16, slog2w=10, c_mult=cm)
    sk.update(_dev(x))
    C2 = oracle.sketch_update(oracle.new_counters(p), p, x)
    C1 = oracle.sketch_update_super(oracle.new_counters(q), p, q, F, x)
    gk, ge = sk.topk(k)
    wk, we = oracle.topk_hier(C2, p, C1, q, F, k, cm, nthreads=NT)
    assert np.array_equal(gk, wk) and np.array_equal(ge, we)
    assert (ge == 0).sum() > 1000


def test_hier_covering_every_super_item_is_flat_search(hs, data):
    F = 8
    k = 300
    cm = (32 ** 3 + k - 1) // k
    sk, p, q = pair(hs, F, c_mult=cm)
    flat = hs.Sketch(5, 14, 25.6, 0.1, 3, 4)
    xd = _dev(data)
    sk.update(xd)
    flat.update(xd)
    a, b = sk.topk(k), flat.topk(k)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_hier_reset_seek_merge(hs, data):
    F = 4
    a, p, q = pair(hs, F)
    b, _, _ = pair(hs, F)
    xd = _dev(data)
    half = len(data) // 2
    a.update(xd[:half])
    b.seek(half)
    b.update(xd[half:])
    a.merge(b)
    whole, _, _ = pair(hs, F)
    whole.update(xd)
    assert np.array_equal(a.counters(), whole.counters())
    assert np.array_equal(a.super_counters(), whole.super_counters())
    ta, tw = a.topk(100), whole.topk(100)
    assert np.array_equal(ta[0], tw[0]) and np.array_equal(ta[1], tw[1])
    a.reset()
    assert not a.counters().any() and not a.super_counters().any()


def test_hier_argument_checks(hs):
    sk = hs.Sketch(5, 12, 25.6, 0.1, 1)
    with pytest.raises(hs.HSError):
        sk.set_hierarchy(7, 10)          # 256 is not a multiple of 7
    sk.update(_dev(np.zeros((10, 3), np.float32)))
    with pytest.raises(hs.HSError):
        sk.set_hierarchy(8, 10)          # not a fresh sketch
