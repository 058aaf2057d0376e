"""The synthetic halo boxes: deterministic, in range, and drawn from the stated laws."""
import numpy as np
import pytest
from scipy import stats

import synth


def test_deterministic_and_thread_independent():
    b = synth.HaloBox(synth.small_box(0))
    x1 = b.generate(0, 50000, nthreads=1)
    x4 = b.generate(0, 50000, nthreads=4)
    assert np.array_equal(x1, x4)
    b2 = synth.HaloBox(synth.small_box(0))
    assert np.array_equal(b2.generate(1000, 3000), x1[1000:4000])
    b3 = synth.HaloBox(synth.small_box(1))
    assert not np.array_equal(b3.generate(0, 1000), x1[:1000])


def test_range_and_counts():
    spec = synth.small_box(0)
    b = synth.HaloBox(spec)
    x = b.generate()
    assert x.dtype == np.float32 and x.shape == (spec.n, 3)
    assert x.min() >= 0.0 and x.max() < spec.box
    assert b.n_in_halos == round(0.7 * spec.n)
    _, _, _, cnt = b.catalogue()
    assert int(cnt.sum()) == b.n_in_halos


def test_stream_order_is_a_permutation():
    spec = synth.BoxSpec(n=12345, box=10.0, n_halo=10, seed=3)
    b = synth.HaloBox(spec)
    idx = np.array([b.stream_index(i) for i in range(spec.n)])
    assert np.array_equal(np.sort(idx), np.arange(spec.n))
    assert not np.array_equal(idx, np.arange(spec.n))


def test_mass_function_power_law():
    spec = synth.BoxSpec(n=1 << 20, box=100.0, n_halo=20000, seed=2)
    _, mass, _, _ = synth.HaloBox(spec).catalogue()
    e = 1.0 - spec.slope
    lo, hi = spec.m_min ** e, spec.m_max ** e
    cdf = lambda m: (np.power(m, e) - lo) / (hi - lo)
    assert stats.kstest(mass, cdf).pvalue > 1e-3
    assert mass.min() >= spec.m_min and mass.max() <= spec.m_max


def test_plummer_radial_profile():
    # one halo, no permutation: its particles are the first n_h of the stream
    spec = synth.BoxSpec(n=200000, box=50.0, n_halo=1, seed=5, halo_frac=0.5, permute=False)
    b = synth.HaloBox(spec)
    centre, _, a, cnt = b.catalogue()
    x = b.generate(0, int(cnt[0])).astype(np.float64)
    d = x - centre[0]
    d -= spec.box * np.round(d / spec.box)               # minimum image
    r = np.sqrt((d * d).sum(1))
    T = spec.trunc
    mt = (T * T / (T * T + 1)) ** 1.5
    cdf = lambda rr: np.minimum((rr * rr / (rr * rr + a[0] ** 2)) ** 1.5 / mt, 1.0)
    # float32 positions limit the radius resolution near the centre
    assert stats.kstest(r[r > 1e-3 * a[0]], lambda rr: (cdf(rr) - cdf(1e-3 * a[0])) /
                        (1 - cdf(1e-3 * a[0]))).pvalue > 1e-3
    assert r.max() <= T * a[0] * (1 + 1e-5)


def test_subvolume_recipe():
    specs = synth.subvolume_specs()
    n = np.array([s.n for s in specs])
    assert len(specs) == 64
    assert n.min() >= 2 ** 16 and n.max() <= 2 ** 26
    assert abs(n.sum() - 3e8) < 0.01 * 3e8
    for s in specs:
        G = round(s.box / 0.1)
        assert abs(G * 0.1 - s.box) < 1e-9
