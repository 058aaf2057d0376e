"""The full search's pruning rules, checked over every cell of small meshes
against the oracle's sketch and estimates (CPU only).

The device search (Algorithm 1's query done as a full search, Sec. 3.1) does
not estimate all G^3 cells.  It relies on three rules, restated here from the
estimator's definition (Sec. 2.2: the median over the t rows of the signed
counts s_r(j) * C[r][b_r(j)], the lower median for even t):

1. a cell whose estimate reaches theta >= 1 has at least
   need = t - floor((t - 1) / 2) rows whose signed count reaches theta
   ("hot" rows of the cell);
2. a row is hot for a cell exactly when the cell's bucket is set in the row's
   map for the cell's sign: the positive map (C >= theta) for s = +1, the
   negative map (C <= -theta) for s = -1;
3. every such cell is hot in one of the first F = t - need + 1 rows; the search
   enumerates the cells hot in row r < F, drops a cell as soon as the rows
   after r can no longer make `need` hot rows, reports it only if the rows
   before r are cold (so from its first hot row), and then estimates it.

Each test plants nothing: it checks that these rules report exactly the cells
whose oracle estimate reaches theta, each once, and that the directory's
interval of line values per (column, bucket, sign) follows from the oracle's
hash.
"""
import numpy as np
import pytest

import oracle


def _clustered(rng, n, box, halos):
    """n positions: half in Gaussian blobs around `halos` centres, half uniform."""
    centres = rng.uniform(0.0, box, size=(halos, 3))
    m = n // 2
    pick = rng.integers(0, halos, size=m)
    blob = centres[pick] + rng.normal(0.0, 0.02 * box, size=(m, 3))
    flat = rng.uniform(0.0, box, size=(n - m, 3))
    xyz = np.concatenate([blob % box, flat]).astype(np.float32)
    return np.ascontiguousarray(xyz)


def _cells(p):
    G = p.G
    return [(cx, cy, cz) for cz in range(G) for cy in range(G) for cx in range(G)]


def _row_tables(C, p, cells):
    """bucket and sign of every cell in every row (the oracle's hash)."""
    t = p.rows
    b = np.empty((len(cells), t), np.int64)
    s = np.empty((len(cells), t), np.int64)
    for i, c in enumerate(cells):
        for r in range(t):
            b[i, r], s[i, r] = oracle.hash_row(p, r, c)
    return b, s


def _search_by_rules(C, b, s, t, theta):
    """Cells (indices) the pruned search reports, with how often each is reported."""
    need = t - (t - 1) // 2
    F = t - need + 1
    pos = C >= theta                                   # positive maps
    neg = C <= -theta                                  # negative maps
    rows = np.arange(t)
    hot = np.where(s > 0, pos[rows, b], neg[rows, b])  # rule 2: cell x row
    reports = {}
    for r in range(F):
        for i in np.nonzero(hot[:, r])[0]:
            nhot, left, dropped = 1, t - 1 - r, False
            for rr in range(r + 1, t):                 # the rows after r, early exit
                nhot += int(hot[i, rr])
                left -= 1
                if nhot + left < need:
                    dropped = True
                    break
            if dropped or nhot < need:
                continue
            if hot[i, :r].any():                       # reported from its first hot row
                continue
            reports[i] = reports.get(i, 0) + 1
    return reports, hot


@pytest.mark.parametrize("rows,log2w,seed", [(5, 6, 1), (5, 9, 2), (3, 5, 3), (4, 6, 4), (6, 7, 5)])
def test_pruned_search_reports_exactly_the_passing_cells(rows, log2w, seed):
    rng = np.random.default_rng(seed)
    p = oracle.Params(rows, log2w, 20.0, 1.0, hash_seed=1000 + seed)
    xyz = _clustered(rng, 40000, 20.0, halos=12)
    C = oracle.new_counters(p)
    oracle.sketch_update(C, p, xyz)
    cells = _cells(p)
    keys = np.array([cx + p.G * (cy + p.G * cz) for cx, cy, cz in cells], np.uint64)
    est = oracle.estimate(C, p, keys)
    b, s = _row_tables(C, p, cells)
    signed = s * C[np.arange(rows), b]                 # s_r * C[r][b_r], cell x row
    assert (np.sort(signed, axis=1)[:, (rows - 1) // 2] == est).all()   # the lower median
    need = rows - (rows - 1) // 2
    top = np.sort(est)[::-1]
    # thresholds: 1, a tie-heavy low value, the estimate of rank 100 and 10, the maximum
    thetas = sorted({1, int(top[2000]) if top[2000] >= 1 else 1, int(max(top[100], 1)),
                     int(max(top[10], 1)), int(max(top[0], 1))})
    for theta in thetas:
        reports, hot = _search_by_rules(C, b, s, rows, theta)
        assert (hot == (signed >= theta)).all()        # rule 2
        passing = set(np.nonzero(est >= theta)[0].tolist())
        assert all(hot[i].sum() >= need for i in passing)   # rule 1
        assert set(reports) == passing                 # rule 3: nothing lost, nothing extra
        assert all(v == 1 for v in reports.values())   # each cell once


def test_negative_counters_make_cells_hot_through_the_negative_map():
    """A sketch where most hot rows are hot by a negative counter and a sign of -1."""
    rng = np.random.default_rng(7)
    p = oracle.Params(5, 4, 12.0, 1.0, hash_seed=77)
    xyz = _clustered(rng, 30000, 12.0, halos=6)
    C = oracle.new_counters(p)
    oracle.sketch_update(C, p, xyz)
    cells = _cells(p)
    keys = np.array([cx + p.G * (cy + p.G * cz) for cx, cy, cz in cells], np.uint64)
    est = oracle.estimate(C, p, keys)
    b, s = _row_tables(C, p, cells)
    theta = int(np.sort(est)[::-1][50])
    assert theta >= 1
    reports, hot = _search_by_rules(C, b, s, 5, theta)
    by_neg = hot & (s < 0)
    assert by_neg.any()                                # the negative maps are exercised
    assert set(reports) == set(np.nonzero(est >= theta)[0].tolist())


@pytest.mark.parametrize("log2w", [4, 13, 24, 26])
def test_bucket_and_sign_of_a_column_is_a_half_interval_of_line_values(log2w):
    """The directory query's interval: in row r, with v = a0 cx + L(cy, cz)
    (mod 2^64) and L(cy, cz) = a1 cy + a2 cz + b, the cells of column cx whose
    (bucket, sign) is (B, s) are the lines with L in
    [h 2^(63 - log2 W) - a0 cx, (h + 1) 2^(63 - log2 W) - a0 cx) (mod 2^64),
    h = B << 1 | (s < 0): the oracle's bucket is the top log2 W bits of v and
    its sign the next bit.  An interval that long covers one or two slots of
    2^(64 - D) values for any D <= log2 W + 1."""
    rng = np.random.default_rng(log2w)
    p = oracle.Params(5, log2w, 64.0, 1.0, hash_seed=31 + log2w)
    M = 1 << 64
    half = 1 << (63 - log2w)
    for r in range(p.rows):
        a0, a1, a2, b = (int(x) for x in p.seeds[4 * r:4 * r + 4])
        for _ in range(200):
            cx, cy, cz = (int(x) for x in rng.integers(0, p.G, size=3))
            B, s = oracle.hash_row(p, r, (cx, cy, cz))
            h = (B << 1) | (1 if s < 0 else 0)
            L = (a1 * cy + a2 * cz + b) % M
            lo = (h * half - a0 * cx) % M
            assert (L - lo) % M < half                        # inside its own interval
            other = h ^ 1                                     # the same bucket, other sign
            assert (L - (other * half - a0 * cx)) % M >= half
            for D in range(1, log2w + 2):
                first = lo >> (64 - D)
                last = ((lo + half - 1) % M) >> (64 - D)
                assert (last - first) % (1 << D) <= 1         # one slot or two
