"""Packed 64-bit particle records on the GPU vs the CPU oracle: the packing
kernel, the update from records (binned and direct, host and device, aligned
and not) and the top-k, bit for bit."""
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
    x = synth.HaloBox(synth.small_box(6)).generate()
    x[10] = [np.nan, 1.0, 1.0]
    x[11] = [100.0, -0.3, 250.0]                         # wraps
    return x


def _pack_gpu(hs, x, box):
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    out = torch.empty(len(x), dtype=torch.int64, device="cuda")
    hs.pack_positions(xd, box, out)
    torch.cuda.synchronize()
    return out


def test_pack_kernel_bitexact(hs, small):
    got = _pack_gpu(hs, small, 100.0).cpu().numpy().view(np.uint64)
    assert np.array_equal(got, oracle.pack(small, 100.0))


FLAGS = {"auto": 0, "direct": 4, "binned": 8}


@pytest.mark.parametrize("rate", [1.0, 0.1])
@pytest.mark.parametrize("update", list(FLAGS))
def test_packed_update_and_topk_bitexact(hs, small, rate, update):
    rec = _pack_gpu(hs, small, 100.0)
    sk = hs.Sketch(5, 16, 100.0, 0.1, 13, 14, flags=FLAGS[update])
    cut = len(small) // 3 + 1                            # the second call starts 8-byte aligned only
    sk.update_packed(rec[:cut], rate=rate)
    sk.update_packed(rec[cut:], rate=rate)
    p = oracle.Params(5, 16, 100.0, 0.1, 13, 14)
    pk = oracle.pack(small, 100.0)
    C = oracle.sketch_update_packed(oracle.new_counters(p), p, pk, rate=rate, nthreads=NT)
    assert np.array_equal(sk.counters(), C)
    keys, est = sk.topk(500)
    wk, we = oracle.topk_full(C, p, 500, nthreads=NT)
    assert np.array_equal(keys, wk) and np.array_equal(est, we)


def test_packed_update_from_host_records(hs, small):
    pk = oracle.pack(small, 100.0)
    sk = hs.Sketch(5, 16, 100.0, 0.1, 3, 4)
    sk.update_packed(pk[:777])
    sk.update_packed(pk[777:])
    p = oracle.Params(5, 16, 100.0, 0.1, 3, 4)
    C = oracle.sketch_update_packed(oracle.new_counters(p), p, pk, nthreads=NT)
    assert np.array_equal(sk.counters(), C)


def test_packed_with_hierarchy(hs):
    x = synth.HaloBox(synth.BoxSpec(n=1 << 18, box=25.6, n_halo=250, seed=8)).generate()
    F, cm, k = 8, 2, 300
    sk = hs.Sketch(5, 14, 25.6, 0.1, 3, 4)
    sk.set_hierarchy(F, 12, cm)
    pk = oracle.pack(x, 25.6)
    sk.update_packed(torch.from_numpy(pk.view(np.int64)).cuda(), rate=0.5)
    p = oracle.Params(5, 14, 25.6, 0.1, 3, 4)
    q = oracle.super_params(p, F, 12)
    C2 = oracle.sketch_update_packed(oracle.new_counters(p), p, pk, rate=0.5, nthreads=NT)
    C1 = oracle.sketch_update_packed(oracle.new_counters(q), q, pk, rate=0.5, F=F, fine=p)
    assert np.array_equal(sk.counters(), C2)
    assert np.array_equal(sk.super_counters(), C1)
    keys, est = sk.topk(k)
    wk, we = oracle.topk_hier(C2, p, C1, q, F, k, cm, nthreads=NT)
    assert np.array_equal(keys, wk) and np.array_equal(est, we)


def test_packed_refused_by_learned_sketch(hs, small):
    L = hs.Learned(3, 14, 100.0, 0.1, coarse_factor=10, table_log2=14)
    L.prepare(torch.from_numpy(small[:1000]).cuda(), hs.MLP())
    with pytest.raises(hs.HSError):
        hs.sketch_update_packed(L.sketch_h, oracle.pack(small[:100], 100.0))
