"""The compaction pass (every particle sampled and quantised once, the kept
cells then read by each scatter pass) against the CPU oracle.

It runs when an update would otherwise read the positions several times: a
hierarchy (Algorithm 3: the sketch and its super-item sketch) at a low sample
rate, and a sketch updated in row passes.  Counters of both layers and the
ranked top-k (whose threshold comes from the probe the compaction writes)
must equal the oracle's bit for bit, from device, page-locked and pageable
host memory."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

NT = oracle.default_threads()
BINNED = 8          # HS_FLAG_UPDATE_BINNED


@pytest.fixture(scope="module")
def hs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_00975_gb300 import halosketch
    halosketch.lib()
    return halosketch


@pytest.fixture(scope="module")
def box():
    spec = synth.BoxSpec(n=6_000_000, box=50.0, n_halo=6000, seed=41)
    return spec, synth.HaloBox(spec).generate()


def _src(x, memory):
    if memory == "device":
        return torch.from_numpy(np.ascontiguousarray(x)).cuda()
    if memory == "pinned":
        return torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
    return np.ascontiguousarray(x)


@pytest.mark.parametrize("memory", ["device", "pinned", "pageable"])
@pytest.mark.parametrize("rate", [0.1, 0.3])
def test_hierarchy_compacted_bitexact(hs, box, memory, rate):
    spec, x = box
    F = 10
    sk = hs.Sketch(5, 20, spec.box, 0.1, 7, 8, flags=BINNED)
    sk.set_hierarchy(F, 18, 2)
    cut = 2_500_001                         # two calls: the index runs on
    sk.update(_src(x[:cut], memory), rate=rate)
    sk.update(_src(x[cut:], memory), rate=rate)
    p = oracle.Params(5, 20, spec.box, 0.1, 7, 8)
    q = oracle.super_params(p, F, 18)
    C = oracle.sketch_update(oracle.new_counters(p), p, x, rate=rate, nthreads=NT)
    S = oracle.sketch_update_super(oracle.new_counters(q), p, q, F, x, rate=rate)
    assert np.array_equal(sk.counters(), C)
    assert np.array_equal(sk.super_counters(), S)
    keys, est = sk.topk(300)
    wk, we = oracle.topk_hier(C, p, S, q, F, 300, 2, nthreads=NT)
    assert np.array_equal(keys, wk) and np.array_equal(est, we)
    sk.close()


@pytest.mark.parametrize("memory", ["device", "pinned"])
def test_row_passes_compacted_bitexact(hs, box, memory):
    """5 x 2^26: the rings of all rows do not fit one block, so the update
    runs in row passes over the compacted cells."""
    spec, x = box
    part = x[:3_000_000]
    sk = hs.Sketch(5, 26, spec.box, 0.1, 9, 10, flags=BINNED)
    sk.update(_src(part, memory), rate=0.1)
    p = oracle.Params(5, 26, spec.box, 0.1, 9, 10)
    C = oracle.sketch_update(oracle.new_counters(p), p, part, rate=0.1, nthreads=NT)
    assert np.array_equal(sk.counters(), C)
    keys, est = sk.topk(200)
    wk, we = oracle.topk_full(C, p, 200, nthreads=NT)
    assert np.array_equal(keys, wk) and np.array_equal(est, we)
    sk.close()


@pytest.mark.parametrize("memory", ["device", "pinned", "pageable"])
def test_packed_records_compacted_bitexact(hs, box, memory):
    """Packed position records (three 21-bit coordinates) at rate 0.1 into a
    hierarchy: each record is decoded and sampled once by the compaction pass,
    then both layers' passes read the kept cells."""
    spec, x = box
    F = 10
    pk = oracle.pack(x, spec.box)
    rec = pk.view(np.int64)
    src = (torch.from_numpy(rec).cuda() if memory == "device" else
           torch.from_numpy(rec).pin_memory() if memory == "pinned" else np.ascontiguousarray(rec))
    sk = hs.Sketch(5, 20, spec.box, 0.1, 7, 8, flags=BINNED)
    sk.set_hierarchy(F, 18, 2)
    sk.update_packed(src, rate=0.1)
    p = oracle.Params(5, 20, spec.box, 0.1, 7, 8)
    q = oracle.super_params(p, F, 18)
    C = oracle.sketch_update_packed(oracle.new_counters(p), p, pk, rate=0.1, nthreads=NT)
    S = oracle.sketch_update_packed(oracle.new_counters(q), q, pk, rate=0.1, F=F, fine=p)
    assert np.array_equal(sk.counters(), C)
    assert np.array_equal(sk.super_counters(), S)
    keys, est = sk.topk(300)
    wk, we = oracle.topk_hier(C, p, S, q, F, 300, 2, nthreads=NT)
    assert np.array_equal(keys, wk) and np.array_equal(est, we)
    sk.close()
