"""Pins of the packed-record oracle (Sec. 4's 64-bit particle records; the
reading: three 21-bit coordinates q = floor(fl32(x * fl32(2^21 / L))), cell
(q * G) >> 21).  Checked against numpy float32 arithmetic, exact integer
arithmetic, the float32 mesh reduction (Sec. 2.1) at cell centres, and the plain
Count Sketch update (Sec. 2.2) by reduction."""
import numpy as np
import pytest

import oracle
import synth

L21 = 1 << 21


def test_pack_layout_and_rounding():
    rng = np.random.default_rng(0)
    L = 100.0
    x = rng.uniform(0, L, (5000, 3)).astype(np.float32)
    x[0] = [0.0, L, -0.25]                        # the edge wraps, negatives wrap
    x[1] = [np.nan, 1.0, 1.0]
    x[2] = [np.inf, 1.0, 1.0]
    p = oracle.pack(x, L)
    s = np.float32(L21 / L)
    with np.errstate(invalid="ignore"):
        q = np.floor((x * s).astype(np.float32)).astype(np.int64) % L21
    want = q[:, 0].astype(np.uint64) | (q[:, 1].astype(np.uint64) << np.uint64(21)) | \
        (q[:, 2].astype(np.uint64) << np.uint64(42))
    ok = np.isfinite(x).all(1)
    assert np.array_equal(p[ok], want[ok])
    assert (p[~ok] == oracle.PACK_INVALID).all() and (~ok).sum() == 2
    assert p[0] & np.uint64(L21 - 1) == 0 and (p[0] >> np.uint64(21)) & np.uint64(L21 - 1) == 0
    assert p[0] >> np.uint64(42) == np.uint64(L21 - int(np.ceil(0.25 * float(s))))


def test_cell_of_packed_is_exact_integer_division():
    rng = np.random.default_rng(1)
    for G in (1, 7, 1000, 5000, 20000, L21):
        for _ in range(200):
            q = [int(v) for v in rng.integers(0, L21, 3)]
            pk = q[0] | (q[1] << 21) | (q[2] << 42)
            assert oracle.cell_packed(pk, G) == tuple(qq * G // L21 for qq in q)
    assert oracle.cell_packed(1 << 63, 5000) is None


def test_packed_cells_equal_float_cells_at_centres_and_nearby_elsewhere():
    p = oracle.Params(1, 8, 100.0, 0.1, 0)
    rng = np.random.default_rng(2)
    c = rng.integers(0, p.G, (3000, 3))
    centres = ((c + 0.5) * 0.1).astype(np.float32)
    pk = oracle.pack(centres, 100.0)
    assert all(oracle.cell_packed(int(v), p.G) == tuple(int(a) for a in cc) for v, cc in zip(pk, c))
    x = synth.HaloBox(synth.small_box(3)).generate(0, 20000)
    pk = oracle.pack(x, 100.0)
    kf = oracle.keys_of(x, p).astype(np.int64)
    cf = np.stack([kf % p.G, (kf // p.G) % p.G, kf // (p.G * p.G)], 1)
    cp = np.array([oracle.cell_packed(int(v), p.G) for v in pk])
    d = (cp - cf + p.G // 2) % p.G - p.G // 2                # periodic difference
    assert np.abs(d).max() <= 1                              # a boundary moves by < 0.25 kpc
    assert (d != 0).any(1).mean() < 0.02


@pytest.mark.parametrize("rate,g0,nt", [(1.0, 0, 1), (0.3, 77, 4)])
def test_packed_update_is_the_update_of_cell_centres(rate, g0, nt):
    x = synth.HaloBox(synth.BoxSpec(n=30000, box=12.8, n_halo=50, seed=4)).generate()
    x[5] = np.nan                                            # an invalid record is skipped
    p = oracle.Params(3, 12, 12.8, 0.1, 9, 10)
    pk = oracle.pack(x, 12.8)
    C = oracle.sketch_update_packed(oracle.new_counters(p), p, pk, g0=g0, rate=rate, nthreads=nt)
    valid = pk != oracle.PACK_INVALID
    cells = np.array([oracle.cell_packed(int(v), p.G) if ok else (0, 0, 0)
                      for v, ok in zip(pk, valid)])
    centres = ((cells + 0.5) * 0.1).astype(np.float32)
    centres[~valid] = np.nan
    want = oracle.sketch_update(oracle.new_counters(p), p, centres, g0=g0, rate=rate)
    assert np.array_equal(C, want) and C.any()
    # the super-item layer: super cells of the packed cells
    F = 8
    q = oracle.super_params(p, F, 10)
    C1 = oracle.sketch_update_packed(oracle.new_counters(q), q, pk, g0=g0, rate=rate, F=F, fine=p)
    sc = ((cells // F + 0.5) * (F * 0.1)).astype(np.float32)
    sc[~valid] = np.nan
    assert np.array_equal(C1, oracle.sketch_update(oracle.new_counters(q), q, sc, g0=g0, rate=rate))
