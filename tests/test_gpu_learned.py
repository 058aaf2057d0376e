"""Learned router on the GPU vs the CPU oracle, through the C ABI.

Bit for bit: coarse sample counts, features, logits (the kernel and the
oracle run the same float32 fma chains on the same bf16 values), the routing
decision, the sketch counters, the exact counts of routed cells and the merged
top-k.  Within float tolerance: the summed gradient against the float64
network.  And the point of the router: at no more memory than a plain sketch,
a trained router gives a higher top-k recall on a held-out box.
"""
import numpy as np
import pytest

import oracle
import oracle.learned as OL
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


def rand_params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    P = np.concatenate([
        rng.uniform(-1, 1, 64 * 27) * np.sqrt(6 / 27) * scale, rng.normal(0, 0.1, 64),
        rng.uniform(-1, 1, 64 * 64) * np.sqrt(6 / 64) * scale, rng.normal(0, 0.1, 64),
        rng.uniform(-1, 1, 64) * np.sqrt(6 / 64) * scale, rng.normal(0, 0.1, 1)])
    return P.astype(np.float32)


def rand_feats(seed, m):
    return OL.feature_of(np.random.default_rng(seed).integers(0, 300, size=(m, 27)))


# ---------------------------------------------------------------- MLP

def test_mlp_init_and_params_roundtrip(hs):
    m = hs.MLP(seed=5)
    P = m.get_params()
    w1, b1, w2, b2, w3, b3 = OL.unpack(P)
    assert not b1.any() and not b2.any() and not b3.any()
    assert np.abs(w1).max() <= np.sqrt(6 / 27) and np.abs(w2).max() <= np.sqrt(6 / 64)
    assert np.std(w1) > 0.2
    Q = rand_params(1)
    m.set_params(Q)
    assert np.array_equal(m.get_params(), Q)
    m2 = hs.MLP(seed=5)
    assert np.array_equal(m2.get_params(), P)          # seeded


@pytest.mark.parametrize("m", [1, 127, 128, 5000 + 37])
def test_mlp_forward_bitexact(hs, m):
    mlp = hs.MLP()
    P = rand_params(2)
    mlp.set_params(P)
    F = rand_feats(3, m)
    want = OL.forward_f32(P, F)
    assert np.array_equal(mlp.forward(F).view(np.uint32), want.view(np.uint32))
    assert np.array_equal(mlp.forward(_dev(F)).view(np.uint32), want.view(np.uint32))


@pytest.mark.parametrize("m", [100, 128 * 7 + 5])
def test_mlp_gradient_vs_float64(hs, m):
    mlp = hs.MLP()
    P = rand_params(4)
    mlp.set_params(P)
    F = rand_feats(5, m)
    rng = np.random.default_rng(6)
    y = (rng.random(m) < 0.3).astype(np.float32)
    w = rng.uniform(0.5, 2.0, m).astype(np.float32)
    g, loss = mlp.gradient(_dev(F), _dev(y), _dev(w))
    l64, g64 = OL.loss_and_grad64(P, OL.bf16_value(F).astype(np.float64), y, w, round_bf16=True)
    assert abs(loss - l64) <= 1e-4 * abs(l64)
    # float32 sums of m terms against float64: relative error of the vector
    assert np.linalg.norm(g - g64) <= 1e-4 * np.linalg.norm(g64)
    big = np.abs(g64) > 1e-3 * np.abs(g64).max()
    assert np.mean(np.abs(g - g64)[big] <= 1e-3 * np.abs(g64[big]) + 1e-5) > 0.99


def test_box_examples_do_not_depend_on_thread_order(hs):
    """Examples of one box come out in coarse-key order, identical on repeats."""
    from paper_1711_00975_gb300 import router
    spec = synth.BoxSpec(n=1 << 20, box=50.0, n_halo=500, seed=17)
    xyz = synth.HaloBox(spec).generate()
    mlp = hs.MLP(seed=2)
    d = _dev(xyz)
    runs = [router.box_examples(d, spec.n, spec.box, 0.1, mlp, k_label=20,
                                feature_rate=1.0 / 8) for _ in range(2)]
    (f0, y0, k0), (f1, y1, k1) = runs
    assert np.all(k0[:-1] < k0[1:])
    assert np.array_equal(k0, k1) and np.array_equal(f0, f1) and np.array_equal(y0, y1)
    assert y0.sum() > 0
    mlp.close()


def test_training_repeats_bit_for_bit(hs):
    """The gradient sums run in a fixed order, so two training runs from the
    same seed on the same examples end with identical parameters."""
    from paper_1711_00975_gb300 import router
    rng = np.random.default_rng(11)
    counts = rng.integers(0, 300, size=(150_000, 27))
    y = ((counts[:, 13] > 250) | (rng.random(counts.shape[0]) < 0.02)).astype(np.float32)
    F = OL.feature_of(counts)
    runs = []
    for _ in range(2):
        mlp = hs.MLP(seed=3)
        losses = router.train(mlp, F, y, epochs=2, batch=65536, lr=1e-3, seed=5)
        runs.append((mlp.get_params(), np.array(losses)))
        g, l = mlp.gradient(_dev(F[:70_001]), _dev(y[:70_001]), _dev(np.ones(70_001, np.float32)))
        runs[-1] += (g, l)
        mlp.close()
    (p0, l0, g0, s0), (p1, l1, g1, s1) = runs
    assert np.array_equal(p0.view(np.uint32), p1.view(np.uint32))
    assert np.array_equal(l0, l1) and s0 == s1
    assert np.array_equal(g0.view(np.uint32), g1.view(np.uint32))


def test_mlp_training_reduces_loss(hs):
    rng = np.random.default_rng(7)
    counts = rng.integers(0, 200, size=(20000, 27))
    y = (counts[:, 13] > 150).astype(np.float32)            # heavy iff the centre is dense
    F = OL.feature_of(counts)
    w = np.ones_like(y)
    mlp = hs.MLP(seed=8)
    Fd, yd, wd = _dev(F), _dev(y), _dev(w)
    losses = [mlp.train_step(Fd, yd, wd, 3e-3) for _ in range(500)]
    assert losses[-1] < 0.5 * losses[0]
    z = mlp.forward(Fd)
    # bf16 features cannot separate counts within ~4 % of the threshold; the
    # majority class alone scores 0.755
    assert np.mean((z > 0) == (y > 0)) > 0.9


# ---------------------------------------------------------------- exact counts

def test_exact_counts_vs_oracle(hs):
    x = synth.HaloBox(synth.small_box(1)).generate()
    keys, cnt = hs.exact_counts(_dev(x), len(x), 100.0, 0.1, 22)
    o = np.argsort(keys)
    p = oracle.Params(1, 8, 100.0, 0.1, 0)
    ek, ec = oracle.exact_counts(x, p)
    assert np.array_equal(keys[o], ek) and np.array_equal(cnt[o], ec.astype(np.int32))
    assert cnt.sum() == len(x)
    with pytest.raises(hs.HSError):
        hs.exact_counts(_dev(x), len(x), 100.0, 0.1, 8)   # 256 slots: the table is full


@pytest.mark.parametrize("log2_slots", [16, 22])
def test_exact_object_topk_query_recall(hs, log2_slots):
    spec = synth.BoxSpec(n=40000 if log2_slots == 16 else 1 << 20, box=100.0, n_halo=300, seed=4)
    x = synth.HaloBox(spec).generate()
    E = hs.Exact(100.0, 0.1, log2_slots)
    xd = _dev(x)
    E.add(xd[: len(x) // 3])                                # two ragged calls
    E.add(xd[len(x) // 3:])
    p = oracle.Params(1, 8, 100.0, 0.1, 0)
    ek, ec = oracle.exact_counts(x, p)
    assert E.size() == ek.size
    for k in (1, 10, 1000, ek.size + 5):
        tk, tc = E.topk(k)
        wk, wc = oracle.exact_topk(ek, ec.astype(np.int32), k)
        assert np.array_equal(tk, wk) and np.array_equal(tc, wc), k
    rng = np.random.default_rng(1)
    q = np.concatenate([ek[rng.choice(ek.size, 500)], rng.integers(0, 10 ** 9, 500).astype(np.uint64)])
    lut = dict(zip(ek.tolist(), ec.tolist()))
    assert np.array_equal(E.query(q), np.array([lut.get(int(v), 0) for v in q], np.int32))
    sk = hs.Sketch(3, 12, 100.0, 0.1, 5)
    sk.update(xd)
    mk = sk.topk(300)[0]
    assert E.recall(mk, 300) == oracle.recall_at_k(mk, ek, ec, 300)
    E.reset()
    assert E.size() == 0


# ---------------------------------------------------------------- learned sketch

def centre_router(thr_count):
    """z = f13 - f(thr): a coarse cell is positive iff its own sample count > thr."""
    P = np.zeros(OL.N_PARAMS, np.float32)
    w1, b1, w2, b2, w3, b3 = OL.unpack(P)
    w1[0, 13] = 1.0
    w2[0, 0] = 1.0
    w3[0] = 1.0
    b3[0] = -OL.bf16_value(OL.feature_of([thr_count]))[0]
    return P


BOX = dict(n=1 << 18, box=25.6, n_halo=250)


@pytest.fixture(scope="module")
def learned_box():
    return synth.HaloBox(synth.BoxSpec(seed=11, **BOX)).generate()


@pytest.mark.parametrize("table_log2,params", [(12, "centre"), (16, "centre"), (14, "random")])
def test_learned_prepare_bitexact(hs, learned_box, table_log2, params):
    x = learned_box
    R, fseed, frate = 8, 99, 0.25
    L = hs.Learned(3, 14, BOX["box"], 0.1, 21, 22, coarse_factor=R, table_log2=table_log2,
                   feature_seed=fseed, feature_rate=frate)
    mlp = hs.MLP(seed=3)
    P = centre_router(4) if params == "centre" else rand_params(9, scale=2.0)
    mlp.set_params(P)
    nr = L.prepare(_dev(x), mlp)
    p = oracle.Params(3, 14, BOX["box"], 0.1, 21, 22)
    counts, okeys, ofeat, ologit, routed = oracle_routing(x, p, R, fseed, frate, P, table_log2)
    assert np.array_equal(L.coarse_counts(), counts)
    ckeys, logits = L.logits()                              # list order is the GPU's own
    o = np.argsort(ckeys)
    assert np.array_equal(ckeys[o], okeys)
    assert np.array_equal(L.features()[o], ofeat)
    assert np.array_equal(logits[o].view(np.uint32), ologit.view(np.uint32))
    B = OL.route_budget(table_log2, R)
    assert L.max_routed == B
    assert np.array_equal(L.routed(), np.flatnonzero(routed).astype(np.uint64))
    assert nr == routed.sum() == min(B, int((ologit > 0).sum()))


def oracle_routing(x, p, R, fseed, frate, P, table_log2):
    """The oracle's routing: sample counts -> features -> logits -> budgeted routing."""
    counts = OL.coarse_hist(x, p, R, fseed, frate)
    Gc = p.G // R
    okeys = np.flatnonzero(counts).astype(np.uint64)
    ofeat = OL.features(counts, Gc, okeys)
    ologit = OL.forward_f32(P, ofeat)
    routed = OL.route_bytes(okeys, ologit, Gc, OL.route_budget(table_log2, R))
    return counts, okeys, ofeat, ologit, routed


@pytest.mark.parametrize("rate", [1.0, 0.5])
@pytest.mark.parametrize("table_log2", [12, 16])
def test_learned_update_and_topk_bitexact(hs, learned_box, rate, table_log2):
    x = learned_box
    R = 8
    L = hs.Learned(5, 14, BOX["box"], 0.1, 31, 32, coarse_factor=R, table_log2=table_log2,
                   feature_seed=7, feature_rate=0.25)
    mlp = hs.MLP()
    P = centre_router(3)
    mlp.set_params(P)
    L.prepare(_dev(x), mlp)
    xd = _dev(x)
    half = len(x) // 2 + 13                                 # two ragged calls
    L.update(xd[:half], rate=rate)
    L.update(xd[half:], rate=rate)
    p = oracle.Params(5, 14, BOX["box"], 0.1, 31, 32)
    routed = oracle_routing(x, p, R, 7, 0.25, P, table_log2)[4]
    assert np.array_equal(L.routed(), np.flatnonzero(routed).astype(np.uint64))
    C = oracle.new_counters(p)
    tk, tc = OL.learned_update(C, p, x, routed, R, rate=rate)
    assert np.array_equal(L.counters(), C)
    gk, gc = L.table()
    assert np.array_equal(gk, tk) and np.array_equal(gc, tc)
    wk, we = OL.learned_topk(C, p, routed, R, tk, tc, 1000)
    for k in (1, 100, 1000):                                # oracle ranking prefixes
        lk, le = L.topk(k)
        assert np.array_equal(lk, wk[:k]) and np.array_equal(le, we[:k]), k
    # reset keeps the routing; the same stream gives the same state
    L.reset()
    assert not L.counters().any() and L.table()[0].size == 0
    L.update(xd, rate=rate)
    assert np.array_equal(L.counters(), C)


def test_learned_empty_routing_equals_plain(hs, learned_box):
    x = learned_box
    L = hs.Learned(5, 14, BOX["box"], 0.1, 41, 0, coarse_factor=8, table_log2=14,
                   feature_seed=1, feature_rate=0.25)
    mlp = hs.MLP()
    P = np.zeros(OL.N_PARAMS, np.float32)
    P[-1] = -1.0                                            # every logit is -1
    mlp.set_params(P)
    assert L.prepare(_dev(x), mlp) == 0
    L.update(_dev(x))
    sk = hs.Sketch(5, 14, BOX["box"], 0.1, 41, 0)
    sk.update(_dev(x))
    assert np.array_equal(L.counters(), sk.counters())
    a, b = L.topk(500), sk.topk(500)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


# ---------------------------------------------------------------- the gain

def test_trained_router_beats_plain_sketch_at_no_more_memory(hs):
    from paper_1711_00975_gb300 import router
    box, cell, R, k = 50.0, 0.1, 10, 100
    mlp = hs.MLP(seed=1)
    feats, ys = [], []
    for seed in range(1000, 1008):                          # training boxes
        x = synth.HaloBox(synth.BoxSpec(n=10 ** 6, box=box, n_halo=1000, seed=seed)).generate()
        f, y, _ = router.box_examples(_dev(x), len(x), box, cell, mlp, R, k_label=k,
                                      log2_slots=22)
        feats.append(f)
        ys.append(y)
    F = np.concatenate(feats)
    Y = np.concatenate(ys)
    assert 0 < Y.sum() < 0.05 * Y.size
    losses = router.train(mlp, F, Y, epochs=40, batch=8192, lr=2e-3, seed=0)
    assert losses[-1] < losses[0]
    # held-out box: plain 5 x 2^14 (320 KiB) vs learned 5 x 2^13 + 2^13-slot table (256 KiB)
    x = synth.HaloBox(synth.BoxSpec(n=10 ** 6, box=box, n_halo=1000, seed=7)).generate()
    xd = _dev(x)
    ek, ec = hs.exact_counts(xd, len(x), box, cell, 22)
    plain = hs.Sketch(5, 14, box, cell, 1)
    plain.update(xd)
    r_plain = oracle.recall_at_k(plain.topk(k)[0], ek, ec, k)
    L = hs.Learned(5, 13, box, cell, 1, coarse_factor=R, table_log2=13)
    L.prepare(xd, mlp)
    L.update(xd)
    r_learned = oracle.recall_at_k(L.topk(k)[0], ek, ec, k)
    mem_plain = 5 * 4 << 14
    mem_learned = (5 * 4 << 13) + L.table_bytes
    print(f"recall@{k}: plain {r_plain:.3f} ({mem_plain} B), learned {r_learned:.3f} "
          f"({mem_learned} B, {L.max_routed} routed cells)")
    assert mem_learned <= mem_plain
    assert r_learned >= r_plain + 0.05


def test_learned_sample_in_pieces_equals_one_pass(hs, learned_box):
    x = learned_box
    R, fseed, frate = 8, 5, 0.25
    P = rand_params(12, scale=2.0)
    mlp = hs.MLP()
    mlp.set_params(P)
    one = hs.Learned(3, 14, BOX["box"], 0.1, 21, 22, coarse_factor=R, table_log2=14,
                     feature_seed=fseed, feature_rate=frate)
    nr1 = one.prepare(_dev(x), mlp)
    pieces = hs.Learned(3, 14, BOX["box"], 0.1, 21, 22, coarse_factor=R, table_log2=14,
                        feature_seed=fseed, feature_rate=frate)
    cut = len(x) // 3 + 5
    pieces.sample(_dev(x[:cut]))
    pieces.sample(np.ascontiguousarray(x[cut:]))            # host memory, staged
    nr2 = pieces.route(mlp)
    p = oracle.Params(3, 14, BOX["box"], 0.1, 21, 22)
    counts = OL.coarse_hist(x, p, R, fseed, frate)
    assert np.array_equal(one.coarse_counts(), counts)
    assert np.array_equal(pieces.coarse_counts(), counts)
    assert nr1 == nr2
    assert np.array_equal(one.routed(), pieces.routed())
    # a second round of sampling starts a new histogram
    pieces.sample(_dev(x[:cut]))
    pieces.route(mlp)
    assert np.array_equal(pieces.coarse_counts(), OL.coarse_hist(x[:cut], p, R, fseed, frate))


@pytest.mark.parametrize("rate", [1.0, 0.5])
def test_learned_with_hierarchy_bitexact(hs, learned_box, rate):
    x = learned_box
    R = F = 8
    cm, slog2w, k = 3, 11, 400
    L = hs.Learned(5, 14, BOX["box"], 0.1, 31, 32, coarse_factor=R, table_log2=14,
                   feature_seed=7, feature_rate=0.25)
    L.set_hierarchy(F, slog2w, cm)
    P = centre_router(3)
    mlp = hs.MLP()
    mlp.set_params(P)
    L.prepare(np.ascontiguousarray(x), mlp)                  # host memory
    cut = len(x) // 2 + 3
    L.update(_dev(x[:cut]), rate=rate)
    L.update(np.ascontiguousarray(x[cut:]), rate=rate)
    p = oracle.Params(5, 14, BOX["box"], 0.1, 31, 32)
    q = oracle.super_params(p, F, slog2w)
    routed = oracle_routing(x, p, R, 7, 0.25, P, 14)[4]
    assert np.array_equal(L.routed(), np.flatnonzero(routed).astype(np.uint64))
    C2 = oracle.new_counters(p)
    tk, tc = OL.learned_update(C2, p, x, routed, R, rate=rate)
    C1 = oracle.sketch_update_super(oracle.new_counters(q), p, q, F, x, rate=rate)
    assert np.array_equal(L.counters(), C2)
    assert np.array_equal(L.super_counters(), C1)
    gk, gc = L.table()
    assert np.array_equal(gk, tk) and np.array_equal(gc, tc)
    lk, le = L.topk(k)
    wk, we = OL.learned_topk_hier(C2, p, C1, q, F, cm, routed, R, tk, tc, k, nthreads=NT)
    assert np.array_equal(lk, wk) and np.array_equal(le, we)
