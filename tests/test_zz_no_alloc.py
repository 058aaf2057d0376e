"""sketch_query_noalloc: point queries for callers that cannot allocate device
memory when they query (another allocator owns the device memory, or a fixed
budget leaves none to spare).  Its results must equal sketch_query's, call
after call, although every call reuses the same static scratch array of the
library.

Collected last on purpose; it also passes when run alone in a fresh process.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_00975_gb300 import halosketch
    halosketch.lib()
    return halosketch


def _sketch(hs, seed, log2w):
    spec = synth.BoxSpec(n=1 << 18, box=100.0, n_halo=300, seed=seed)
    xyz = synth.HaloBox(spec).generate()
    sk = hs.Sketch(5, log2w, spec.box, 0.1, hash_seed=seed, sample_seed=seed + 1)
    sk.update(torch.from_numpy(xyz).cuda(), rate=0.5)
    rng = np.random.default_rng(seed)
    keys = rng.integers(0, sk.n_cells, 60000, dtype=np.uint64)
    # include occupied cells so most estimates are non-zero
    cells = (np.floor(xyz[:20000].astype(np.float32) * np.float32(10.0)).astype(np.int64) % 1000)
    occ = (cells[:, 0] + 1000 * (cells[:, 1] + 1000 * cells[:, 2])).astype(np.uint64)
    return sk, np.concatenate([keys, occ])


def test_noalloc_query_equals_sketch_query_on_consecutive_calls(hs):
    a, keys_a = _sketch(hs, 3, 16)
    b, keys_b = _sketch(hs, 8, 12)
    want_a = a.query(keys_a)
    want_b = b.query(keys_b)
    assert want_a.any() and want_b.any()
    for _ in range(2):                      # two calls in a row, alternating sketches
        for sk, keys, want in ((a, keys_a, want_a), (b, keys_b, want_b)):
            est = np.full(keys.size, -7, np.int32)
            hs.sketch_query_noalloc(sk.h, keys, est)          # host arrays
            assert np.array_equal(est, want)
            dkeys = torch.from_numpy(keys).cuda()
            dest = torch.full((keys.size,), -7, dtype=torch.int32, device="cuda")
            hs.sketch_query_noalloc(sk.h, dkeys, dest)        # device arrays
            assert np.array_equal(dest.cpu().numpy(), want)
    a.close()
    b.close()


def test_noalloc_query_limits_and_bad_keys(hs):
    sk, keys = _sketch(hs, 5, 14)
    too_many = np.zeros(hs.HS_NOALLOC_QUERY_MAX + 1, np.uint64)
    with pytest.raises(hs.HSError) as e:
        hs.sketch_query_noalloc(sk.h, too_many, np.empty(too_many.size, np.int32))
    assert e.value.status == hs.HS_ERR_ARG
    bad = keys[:100].copy()
    bad[17] = np.uint64(sk.n_cells)
    est = np.full(bad.size, -7, np.int32)
    with pytest.raises(hs.HSError):
        hs.sketch_query_noalloc(sk.h, bad, est)
    want = sk.query(np.delete(bad, 17))
    assert est[17] == 0 and np.array_equal(np.delete(est, 17), want)
    # the flag of the failed call does not leak into the next one
    est2 = np.empty(99, np.int32)
    hs.sketch_query_noalloc(sk.h, np.delete(bad, 17), est2)
    assert np.array_equal(est2, want)
    sk.close()


def test_noalloc_query_at_the_limit_and_with_mixed_arrays(hs):
    sk, keys = _sketch(hs, 11, 15)
    rng = np.random.default_rng(11)
    m = hs.HS_NOALLOC_QUERY_MAX
    full = np.concatenate([keys, rng.integers(0, sk.n_cells, m - keys.size, dtype=np.uint64)])
    assert full.size == m
    want = sk.query(full)
    for _ in range(2):
        est = np.full(m, -7, np.int32)
        hs.sketch_query_noalloc(sk.h, full, est)              # exactly the maximum
        assert np.array_equal(est, want)
    part = full[:70000]
    # host keys with a device est, and device keys with a host est
    dest = torch.full((part.size,), -7, dtype=torch.int32, device="cuda")
    hs.sketch_query_noalloc(sk.h, part, dest)
    assert np.array_equal(dest.cpu().numpy(), want[:part.size])
    hest = np.full(part.size, -7, np.int32)
    hs.sketch_query_noalloc(sk.h, torch.from_numpy(part).cuda(), hest)
    assert np.array_equal(hest, want[:part.size])
    sk.close()
