"""Pins of the learned-router oracle (CPU only).

The router is not part of arXiv:1711.00975 (which uses the Count Sketch
alone); these tests pin the oracle's statement of it against independent
definitions: torch's own bf16 conversion and autograd, central finite
differences, brute-force loops, and reductions to the plain Count Sketch
oracle (Sec. 2.2, Algorithm 1) and the exact algorithm (Sec. 4.2).
"""
import numpy as np
import pytest
import torch

import oracle
import oracle.learned as OL


def rand_params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    w1, b1, w2, b2, w3, b3 = OL.unpack(np.zeros(OL.N_PARAMS))
    P = np.concatenate([
        rng.uniform(-1, 1, w1.size) * np.sqrt(6 / 27) * scale,
        rng.normal(0, 0.1, 64),
        rng.uniform(-1, 1, w2.size) * np.sqrt(6 / 64) * scale,
        rng.normal(0, 0.1, 64),
        rng.uniform(-1, 1, 64) * np.sqrt(6 / 64) * scale,
        rng.normal(0, 0.1, 1),
    ]).astype(np.float32)
    assert P.size == OL.N_PARAMS == 6017
    return P


def rand_feats(seed, m):
    rng = np.random.default_rng(seed)
    return OL.feature_of(rng.integers(0, 200, size=(m, 27)))


# ---- bf16 ----

def test_bf16_matches_torch_and_c():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(0, 1, 20000), rng.normal(0, 1e-30, 100),
                        rng.normal(0, 1e30, 100), [0.0, -0.0, 1.0, 1.00390625, 1.01171875]])
    x = x.astype(np.float32)
    ours = OL.bf16_bits(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(ours, ref)
    lib = oracle._load()
    assert all(lib.or_bf16(float(v)) == int(b) for v, b in zip(x[:2000], ours[:2000]))
    # ties to even: 1 + 2^-8 is halfway between 1 and 1 + 2^-7
    assert OL.bf16_bits(np.float32([1.00390625]))[0] == 0x3F80
    assert OL.bf16_bits(np.float32([1.01171875]))[0] == 0x3F82


def test_feature_closed_forms():
    # log10(1 + n) = 0, 1, 2, 3 exactly at n = 0, 9, 99, 999
    assert list(OL.feature_of([0, 9, 99, 999])) == [0x0000, 0x3F80, 0x4000, 0x4040]
    lib = oracle._load()
    for n in [0, 1, 2, 7, 63, 64, 1000, 65535, 65536, 10 ** 6]:
        assert lib.or_feature_of(n) == OL.feature_of([n])[0]


# ---- features ----

def test_features_brute_force_with_periodic_wrap():
    rng = np.random.default_rng(1)
    Gc = 5
    counts = rng.integers(0, 50, Gc ** 3).astype(np.int32)
    keys = np.array([0, 4, 24, 124, 62, 100], np.uint64)   # corners and faces wrap
    f = OL.features(counts, Gc, keys)
    for s, k in enumerate(keys.tolist()):
        x, y, z = k % Gc, (k // Gc) % Gc, k // (Gc * Gc)
        i = 0
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    c = counts[(x + dx) % Gc + Gc * (((y + dy) % Gc) + Gc * ((z + dz) % Gc))]
                    assert f[s, i] == OL.feature_of([c])[0], (k, dx, dy, dz)
                    i += 1
    # the centre feature is the cell's own count
    assert np.array_equal(f[:, 13], OL.feature_of(counts[keys.astype(np.int64)]))


def test_coarse_hist_is_bincount_of_sampled_coarse_keys():
    import synth
    x = synth.HaloBox(synth.small_box(5)).generate(0, 50000)
    p = oracle.Params(1, 8, 100.0, 0.1, 1)
    R = 10
    Gc = p.G // R
    rate, seed, g0 = 0.25, 77, 123
    h = OL.coarse_hist(x, p, R, seed, rate, g0)
    keys = oracle.keys_of(x, p).astype(np.int64)
    keep = oracle.keep_mask(g0, len(x), seed, rate)
    cx, cy, cz = keys % p.G, (keys // p.G) % p.G, keys // (p.G * p.G)
    ck = cx // R + Gc * (cy // R + Gc * (cz // R))
    ref = np.bincount(ck[keep], minlength=Gc ** 3)
    assert np.array_equal(h, ref)
    assert 0.2 * len(x) < h.sum() < 0.3 * len(x)
    # rate 1 keeps everything
    assert OL.coarse_hist(x, p, R, seed, 1.0, g0).sum() == len(x)


# ---- MLP ----

def torch_forward(P, X, round_bf16):
    w1, b1, w2, b2, w3, b3 = [torch.tensor(np.asarray(a, np.float64)) for a in OL.unpack(P)]
    if round_bf16:
        w1, b1, w2, b2, w3, b3 = [a.float().bfloat16().double() for a in (w1, b1, w2, b2, w3, b3)]
    X = torch.tensor(X, dtype=torch.float64)
    h1 = torch.nn.functional.linear(X, w1, b1).relu()
    if round_bf16:
        h1 = h1.float().bfloat16().double()
    h2 = torch.nn.functional.linear(h1, w2, b2).relu()
    if round_bf16:
        h2 = h2.float().bfloat16().double()
    return torch.nn.functional.linear(h2, w3[None, :], b3).squeeze(1).numpy()


@pytest.mark.parametrize("rb", [False, True])
def test_forward64_matches_torch_layers(rb):
    P = rand_params(2)
    X = OL.bf16_value(rand_feats(3, 300)).astype(np.float64)
    z, _ = OL.forward64(P, X, rb)
    assert np.allclose(z, torch_forward(P, X, rb), rtol=1e-12, atol=1e-12)


def test_forward_f32_close_to_float64_network():
    P = rand_params(4)
    F = rand_feats(5, 2000)
    z32 = OL.forward_f32(P, F)
    z64, _ = OL.forward64(P, OL.bf16_value(F).astype(np.float64), True)
    # float32 accumulation of <= 64 terms of |value| < ~50; hidden bf16 rounding
    # can flip on near-ties, so compare in bulk and allow a few outliers
    err = np.abs(z32 - z64)
    assert np.median(err) < 1e-5
    assert np.mean(err < 1e-3 * (1 + np.abs(z64))) > 0.99


def test_forward_f32_special_weights():
    # w3 picks hidden unit 0 of layer 2, which picks hidden unit 0 of layer 1,
    # which picks input 13 (the centre): z = feature_13 + b3 exactly
    P = np.zeros(OL.N_PARAMS, np.float32)
    w1, b1, w2, b2, w3, b3 = OL.unpack(P)
    w1[0, 13] = 1.0
    w2[0, 0] = 1.0
    w3[0] = 1.0
    b3[0] = -0.5
    F = rand_feats(6, 50)
    z = OL.forward_f32(P, F)
    assert np.array_equal(z, OL.bf16_value(F[:, 13]) - np.float32(0.5))
    # a negative pre-activation is clipped by the ReLU
    w1[0, 13] = -1.0
    assert np.all(OL.forward_f32(P, F) == np.float32(-0.5))


def test_gradient_matches_finite_differences():
    P = rand_params(7).astype(np.float64)
    X = OL.bf16_value(rand_feats(8, 40)).astype(np.float64)
    rng = np.random.default_rng(9)
    y = (rng.random(40) < 0.3).astype(np.float64)
    w = rng.uniform(0.5, 2.0, 40)
    loss, g = OL.loss_and_grad64(P, X, y, w, round_bf16=False)
    idx = np.concatenate([rng.choice(1728, 20, replace=False), 1728 + np.arange(0, 64, 9),
                          1792 + rng.choice(4096, 20, replace=False), 5888 + np.arange(0, 64, 9),
                          5952 + np.arange(0, 64, 7), [6016]])
    h = 1e-6
    for i in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        lp, _ = OL.loss_and_grad64(Pp, X, y, w, round_bf16=False)
        lm, _ = OL.loss_and_grad64(Pm, X, y, w, round_bf16=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_gradient_matches_torch_autograd():
    P = rand_params(10).astype(np.float64)
    X = OL.bf16_value(rand_feats(11, 64)).astype(np.float64)
    rng = np.random.default_rng(12)
    y = (rng.random(64) < 0.5).astype(np.float64)
    w = rng.uniform(0.1, 3.0, 64)
    loss, g = OL.loss_and_grad64(P, X, y, w, round_bf16=False)
    Pt = torch.tensor(P, requires_grad=True)
    o = 0
    parts = []
    for shape in [(64, 27), (64,), (64, 64), (64,), (64,), (1,)]:
        n = int(np.prod(shape))
        parts.append(Pt[o:o + n].reshape(shape))
        o += n
    w1, b1, w2, b2, w3, b3 = parts
    Xt = torch.tensor(X)
    z = torch.nn.functional.linear(torch.nn.functional.linear(
        torch.nn.functional.linear(Xt, w1, b1).relu(), w2, b2).relu(), w3[None, :], b3).squeeze(1)
    lt = torch.nn.functional.binary_cross_entropy_with_logits(
        z, torch.tensor(y), weight=torch.tensor(w), reduction="sum")
    lt.backward()
    assert abs(lt.item() - loss) < 1e-9 * max(1, abs(loss))
    assert np.allclose(Pt.grad.numpy(), g, rtol=1e-9, atol=1e-12)


# ---- routing, learned update and top-k ----

def test_route_budget_and_ties():
    Gc = 4
    keys = np.array([5, 3, 9, 12, 40, 7], np.uint64)
    logits = np.float32([0.5, 2.0, 0.5, -1.0, 0.0, 3.0])
    r = OL.route_bytes(keys, logits, Gc)
    assert set(np.flatnonzero(r).tolist()) == {5, 3, 9, 7}          # logit > 0 only
    r2 = OL.route_bytes(keys, logits, Gc, budget=3)
    assert set(np.flatnonzero(r2).tolist()) == {7, 3, 5}            # 0.5 tie: key 5 before 9
    assert OL.route_budget(20, 10) == (3 << 20) // 1000 == 3145


def small_case(seed=0, n=30000):
    import synth
    x = synth.HaloBox(synth.BoxSpec(n=n, box=6.4, n_halo=40, seed=seed)).generate()
    p = oracle.Params(3, 10, 6.4, 0.1, 11, 5)
    return x, p


def test_learned_update_reduces_to_plain_and_exact():
    x, p = small_case()
    R = 8
    Gc = p.G // R
    # nothing routed: the sketch of all particles, an empty table
    C = oracle.new_counters(p)
    k, c = OL.learned_update(C, p, x, np.zeros(Gc ** 3, np.uint8), R)
    assert k.size == 0
    assert np.array_equal(C, oracle.sketch_update(oracle.new_counters(p), p, x))
    # everything routed: exact counts, an untouched sketch
    C = oracle.new_counters(p)
    k, c = OL.learned_update(C, p, x, np.ones(Gc ** 3, np.uint8), R)
    ek, ec = oracle.exact_counts(x, p)
    assert not C.any()
    assert np.array_equal(k, ek) and np.array_equal(c, ec.astype(np.int32))


def test_learned_update_split_with_sampling():
    x, p = small_case(1)
    R = 8
    Gc = p.G // R
    rng = np.random.default_rng(3)
    routed = (rng.random(Gc ** 3) < 0.3).astype(np.uint8)
    rate, g0 = 0.5, 1000
    C = oracle.new_counters(p)
    k, c = OL.learned_update(C, p, x, routed, R, g0=g0, rate=rate)
    keys = oracle.keys_of(x, p).astype(np.int64)
    keep = oracle.keep_mask(g0, len(x), p.sample_seed, rate)
    cx, cy, cz = keys % p.G, (keys // p.G) % p.G, keys // (p.G * p.G)
    rt = routed[cx // R + Gc * (cy // R + Gc * (cz // R))].astype(bool)
    uk, uc = np.unique(keys[keep & rt], return_counts=True)
    assert np.array_equal(k, uk.astype(np.uint64)) and np.array_equal(c, uc)
    # the sketch holds exactly the kept, unrouted particles: particles outside
    # that set are moved out of the box (skipped), so sampling indices stay put
    y = x.copy()
    y[~(keep & ~rt)] = np.nan
    C2 = oracle.sketch_update(oracle.new_counters(p), p, y, g0=g0, rate=rate)
    assert np.array_equal(C, C2)


def test_topk_unrouted_brute_force():
    x, p = small_case(2)
    R = 8
    Gc = p.G // R
    rng = np.random.default_rng(4)
    routed = (rng.random(Gc ** 3) < 0.2).astype(np.uint8)
    C = oracle.sketch_update(oracle.new_counters(p), p, x)
    kk, ke = OL.learned_topk(C, p, routed, R, np.zeros(0, np.uint64), np.zeros(0, np.int32), 50)
    allk = np.arange(p.n_cells, dtype=np.uint64)
    est = oracle.estimate(C, p, allk).astype(np.int64)
    cx, cy, cz = (allk % p.G).astype(np.int64), ((allk // p.G) % p.G).astype(np.int64), \
        (allk // (p.G * p.G)).astype(np.int64)
    ok = routed[cx // R + Gc * (cy // R + Gc * (cz // R))] == 0
    order = np.lexsort((allk[ok], -est[ok]))[:50]
    assert np.array_equal(kk, allk[ok][order]) and np.array_equal(ke, est[ok][order])
    # no routing: the plain full search
    fk, fe = oracle.topk_full(C, p, 50)
    nk, ne = OL.learned_topk(C, p, np.zeros(Gc ** 3, np.uint8), R, np.zeros(0, np.uint64),
                             np.zeros(0, np.int32), 50)
    assert np.array_equal(fk, nk) and np.array_equal(fe, ne)


def test_threaded_forms_equal_single_threaded():
    P = rand_params(21)
    F = rand_feats(22, 3001)
    assert np.array_equal(OL.forward_f32(P, F).view(np.uint32),
                          OL.forward_f32(P, F, nthreads=4).view(np.uint32))
    x, p = small_case(5)
    R = 8
    Gc = p.G // R
    routed = (np.random.default_rng(7).random(Gc ** 3) < 0.25).astype(np.uint8)
    C1, C4 = oracle.new_counters(p), oracle.new_counters(p)
    a = OL.learned_update(C1, p, x, routed, R, g0=3, rate=0.7)
    b = OL.learned_update(C4, p, x, routed, R, g0=3, rate=0.7, nthreads=4)
    assert np.array_equal(C1, C4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
