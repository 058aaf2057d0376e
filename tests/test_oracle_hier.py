"""Pins of the hierarchical query oracle (Algorithm 3, CSHi) on the CPU.

The super-item sketch is pinned by reduction to the plain update (Sec. 2.2):
adding each particle's super-item equals adding a particle at the centre of
that super-item on a mesh F times coarser.  The query is pinned by brute
force over tiny dictionaries and by its limit: with c*k covering every
super-item it is the full search (Algorithm 1)."""
import numpy as np
import pytest

import oracle
import synth


def box(seed=0, n=40000, L=12.8, halos=60):
    return synth.HaloBox(synth.BoxSpec(n=n, box=L, n_halo=halos, seed=seed)).generate()


@pytest.mark.parametrize("F,rate", [(4, 1.0), (8, 0.5), (1, 1.0)])
def test_super_update_is_update_of_super_centres(F, rate):
    x = box(1)
    p = oracle.Params(3, 12, 12.8, 0.1, 7, 9)
    q = oracle.super_params(p, F, 11)
    C1 = oracle.sketch_update_super(oracle.new_counters(q), p, q, F, x, g0=5, rate=rate)
    keys = oracle.keys_of(x, p).astype(np.int64)
    c = np.stack([keys % p.G, (keys // p.G) % p.G, keys // (p.G * p.G)], 1) // F
    centres = ((c + 0.5) * (F * 0.1)).astype(np.float32)
    assert np.array_equal(oracle.keys_of(centres, q).astype(np.int64),
                          c[:, 0] + q.G * (c[:, 1] + q.G * c[:, 2]))
    want = oracle.sketch_update(oracle.new_counters(q), q, centres, g0=5, rate=rate)
    assert np.array_equal(C1, want)
    assert C1.any()


def test_hier_topk_brute_force():
    x = box(2)
    F = 4
    p = oracle.Params(3, 10, 12.8, 0.1, 3, 0)
    q = oracle.super_params(p, F, 9)
    C2 = oracle.sketch_update(oracle.new_counters(p), p, x)
    C1 = oracle.sketch_update_super(oracle.new_counters(q), p, q, F, x)
    k, cm = 40, 3
    hk, he = oracle.topk_hier(C2, p, C1, q, F, k, cm)
    # brute force: every super-item, the c*k best, every cell inside, the k best
    sk = np.arange(q.n_cells, dtype=np.uint64)
    se = oracle.estimate(C1, q, sk).astype(np.int64)
    top_s = sk[np.lexsort((sk, -se))[:cm * k]].astype(np.int64)
    sx, sy, sz = top_s % q.G, (top_s // q.G) % q.G, top_s // (q.G * q.G)
    l = np.arange(F ** 3)
    lx, ly, lz = l % F, (l // F) % F, l // (F * F)
    cx = (sx[:, None] * F + lx[None, :]).ravel()
    cy = (sy[:, None] * F + ly[None, :]).ravel()
    cz = (sz[:, None] * F + lz[None, :]).ravel()
    fk = (cx + p.G * (cy + p.G * cz)).astype(np.uint64)
    assert np.unique(fk).size == fk.size == cm * k * F ** 3
    fe = oracle.estimate(C2, p, fk).astype(np.int64)
    o = np.lexsort((fk, -fe))[:k]
    assert np.array_equal(hk, fk[o]) and np.array_equal(he, fe[o])
    # the heaviest super-item holds the heaviest cell here
    assert he[0] == oracle.topk_full(C2, p, 1)[1][0]


def test_hier_with_every_super_item_is_the_full_search():
    x = box(3, n=20000, L=6.4, halos=30)
    F = 8
    p = oracle.Params(5, 11, 6.4, 0.1, 13, 0)
    q = oracle.super_params(p, F, 6)
    C2 = oracle.sketch_update(oracle.new_counters(p), p, x)
    C1 = oracle.sketch_update_super(oracle.new_counters(q), p, q, F, x)
    k = 200
    cm = (q.n_cells + k - 1) // k                          # c*k >= (G/F)^3
    hk, he = oracle.topk_hier(C2, p, C1, q, F, k, cm)
    fk, fe = oracle.topk_full(C2, p, k)
    assert np.array_equal(hk, fk) and np.array_equal(he, fe)


def test_hier_unrouted_reductions_and_brute_force():
    import oracle.learned as OL
    x = box(4)
    F = R = 4
    p = oracle.Params(3, 11, 12.8, 0.1, 5, 0)
    q = oracle.super_params(p, F, 9)
    Gc = p.G // R
    rng = np.random.default_rng(6)
    routed = (rng.random(Gc ** 3) < 0.15).astype(np.uint8)
    C2 = oracle.new_counters(p)
    tk, tc = OL.learned_update(C2, p, x, routed, R)
    C1 = oracle.sketch_update_super(oracle.new_counters(q), p, q, F, x)
    k, cm = 60, 3
    # nothing routed: the plain hierarchical query
    none = np.zeros(Gc ** 3, np.uint8)
    a = OL.learned_topk_hier(C2, p, C1, q, F, cm, none, R, [], [], k)
    b = oracle.topk_hier(C2, p, C1, q, F, k, cm)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    # brute force with routing
    sk = np.arange(q.n_cells, dtype=np.uint64)
    se = oracle.estimate(C1, q, sk).astype(np.int64)
    top_s = sk[np.lexsort((sk, -se))[:cm * k]].astype(np.int64)
    sx, sy, sz = top_s % q.G, (top_s // q.G) % q.G, top_s // (q.G * q.G)
    l = np.arange(F ** 3)
    cx = (sx[:, None] * F + (l % F)[None, :]).ravel()
    cy = (sy[:, None] * F + ((l // F) % F)[None, :]).ravel()
    cz = (sz[:, None] * F + (l // (F * F))[None, :]).ravel()
    keep = routed[cx // R + Gc * (cy // R + Gc * (cz // R))] == 0
    fk = (cx + p.G * (cy + p.G * cz)).astype(np.uint64)[keep]
    fe = oracle.estimate(C2, p, fk).astype(np.int64)
    allk = np.concatenate([fk, tk])
    alle = np.concatenate([fe, tc.astype(np.int64)])
    o = np.lexsort((allk, -alle))[:k]
    hk, he = OL.learned_topk_hier(C2, p, C1, q, F, cm, routed, R, tk, tc, k)
    assert np.array_equal(hk, allk[o]) and np.array_equal(he, alle[o])
    # c*k covering every super-item: the flat search over unrouted cells
    cm_all = (q.n_cells + k - 1) // k
    hk, he = OL.learned_topk_hier(C2, p, C1, q, F, cm_all, routed, R, tk, tc, k)
    fk2, fe2 = OL.learned_topk(C2, p, routed, R, tk, tc, k)
    assert np.array_equal(hk, fk2) and np.array_equal(he, fe2)
