"""Oracle of the learned router (TEST INFRASTRUCTURE ONLY).

The router is an addition to arXiv:1711.00975 (which finds heavy cells with the
Count Sketch alone): coarse sample counts -> 27 neighbourhood features ->
MLP 27 -> 64 -> 64 -> 1 -> route a coarse cell iff logit > 0 -> exact counts
for routed fine cells, Count Sketch for the rest.

Two statements of the network:
- `forward_f32` (C, hs_oracle.c): the kernel's precision - bf16 weights,
  inputs and hidden activations, float32 fmaf chains in index order - so the
  routing decision (logit > 0) can be compared bit for bit;
- `forward64` / `backward64` (numpy float64): the textbook network, optionally
  with the same bf16 roundings, for gradient checks (its own gradient is pinned
  by central finite differences).
"""
from __future__ import annotations

import numpy as np

from . import _load, _ptr

MLP_IN, MLP_H = 27, 64
N_PARAMS = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1


def unpack(P):
    P = np.asarray(P)
    o = 0
    w1 = P[o:o + MLP_H * MLP_IN].reshape(MLP_H, MLP_IN); o += MLP_H * MLP_IN
    b1 = P[o:o + MLP_H]; o += MLP_H
    w2 = P[o:o + MLP_H * MLP_H].reshape(MLP_H, MLP_H); o += MLP_H * MLP_H
    b2 = P[o:o + MLP_H]; o += MLP_H
    w3 = P[o:o + MLP_H]; o += MLP_H
    b3 = P[o:o + 1]
    return w1, b1, w2, b2, w3, b3


def bf16_bits(x) -> np.ndarray:
    """float32 -> bf16 bit patterns, round to nearest, ties to even (numpy)."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = u + 0x7FFF + ((u >> 16) & 1)
    return (u >> 16).astype(np.uint16)


def bf16_value(bits) -> np.ndarray:
    return (np.asarray(bits, np.uint16).astype(np.uint32) << 16).view(np.float32)


def bf16_round(x) -> np.ndarray:
    return bf16_value(bf16_bits(x))


def feature_of(n) -> np.ndarray:
    """bf16(float32(log10(1 + n))) of counts n."""
    return bf16_bits(np.log10(1.0 + np.asarray(n, np.float64)).astype(np.float32))


def coarse_hist(xyz, p, R: int, feature_seed: int, feature_rate: float, g0: int = 0) -> np.ndarray:
    Gc = p.G // R
    out = np.zeros(Gc ** 3, np.int32)
    xyz = np.ascontiguousarray(xyz, np.float32)
    _load().or_coarse_hist(_ptr(xyz), xyz.size // 3, g0, p.inv_cell, p.G, R, feature_seed,
                           feature_rate, _ptr(out))
    return out


def features(counts, Gc: int, keys) -> np.ndarray:
    keys = np.ascontiguousarray(keys, np.uint64)
    out = np.empty((keys.size, MLP_IN), np.uint16)
    counts = np.ascontiguousarray(counts, np.int32)
    _load().or_features(_ptr(counts), Gc, _ptr(keys), keys.size, _ptr(out))
    return out


def forward_f32(P, feats, nthreads: int = 1) -> np.ndarray:
    P = np.ascontiguousarray(P, np.float32)
    feats = np.ascontiguousarray(feats, np.uint16)
    m = feats.size // MLP_IN
    out = np.empty(m, np.float32)
    if nthreads > 1:
        _load().or_mlp_forward_f32_mt(_ptr(P), _ptr(feats), m, _ptr(out), nthreads)
    else:
        _load().or_mlp_forward_f32(_ptr(P), _ptr(feats), m, _ptr(out))
    return out


def forward64(P, X, round_bf16: bool = True):
    """(z, cache) of the float64 network on float64 inputs X (m x 27)."""
    w1, b1, w2, b2, w3, b3 = [np.asarray(a, np.float64) for a in unpack(P)]
    if round_bf16:
        w1, b1, w2, b2, w3, b3 = [bf16_round(a.astype(np.float32)).astype(np.float64)
                                  for a in (w1, b1, w2, b2, w3, b3)]
    a1 = X @ w1.T + b1
    h1 = np.maximum(a1, 0.0)
    if round_bf16:
        h1 = bf16_round(h1.astype(np.float32)).astype(np.float64)
    a2 = h1 @ w2.T + b2
    h2 = np.maximum(a2, 0.0)
    if round_bf16:
        h2 = bf16_round(h2.astype(np.float32)).astype(np.float64)
    z = h2 @ w3 + b3[0]
    return z, (X, a1, h1, a2, h2, w2, w3)


def loss_and_grad64(P, X, y, w, round_bf16: bool = True):
    """Summed loss sum(w (softplus(z) - y z)) and its gradient (the bf16
    roundings pass gradients unchanged)."""
    z, (X, a1, h1, a2, h2, w2, w3) = forward64(P, X, round_bf16)
    y = np.asarray(y, np.float64)
    w = np.asarray(w, np.float64)
    loss = float(np.sum(w * (np.logaddexp(0.0, z) - y * z)))
    dz = w * (1.0 / (1.0 + np.exp(-z)) - y)
    gw3 = h2.T @ dz
    gb3 = np.array([dz.sum()])
    d2 = (dz[:, None] * w3[None, :]) * (a2 > 0)
    gw2 = d2.T @ h1
    gb2 = d2.sum(0)
    d1 = (d2 @ w2) * (a1 > 0)
    gw1 = d1.T @ X
    gb1 = d1.sum(0)
    return loss, np.concatenate([gw1.ravel(), gb1, gw2.ravel(), gb2, gw3, gb3])


def route_budget(table_log2: int, R: int) -> int:
    """Coarse cells the exact part can hold: 12-byte slots -> R^3 int32 counters."""
    return (3 << table_log2) // R ** 3


def route_bytes(keys, logits, Gc: int, budget: int | None = None) -> np.ndarray:
    """One byte per coarse cell: 1 iff its logit > 0 and it is among the
    `budget` cells of largest logit (ties: smaller key first)."""
    keys = np.asarray(keys, np.int64)
    logits = np.asarray(logits, np.float32)
    pos = np.flatnonzero(logits > 0)
    pos = pos[np.lexsort((keys[pos], -logits[pos].astype(np.float64)))]
    if budget is not None:
        pos = pos[:budget]
    r = np.zeros(Gc ** 3, np.uint8)
    r[keys[pos]] = 1
    return r


def learned_update(C, p, xyz, routed, R: int, g0: int = 0, rate: float = 1.0,
                   nthreads: int = 1, cap: int | None = None):
    """Routed particles -> exact table (sorted (keys, counts)); others -> C."""
    xyz = np.ascontiguousarray(xyz, np.float32)
    n = xyz.size // 3
    cap = n + 1 if cap is None else cap
    keys = np.empty(cap, np.uint64)
    cnt = np.empty(cap, np.uint32)
    routed = np.ascontiguousarray(routed, np.uint8)
    D = _load().or_learned_update_mt(_ptr(C), p.rows, p.log2_width, _ptr(p.seeds), _ptr(xyz), n,
                                     g0, p.inv_cell, p.G, p.sample_seed, rate, _ptr(routed), R,
                                     _ptr(keys), _ptr(cnt), cap, nthreads)
    assert D <= cap, "raise cap"
    return keys[:D].copy(), cnt[:D].astype(np.int32)


def learned_topk(C, p, routed, R: int, table_keys, table_counts, k: int):
    """k best of: sketch estimates of cells not routed, exact counts of the table."""
    routed = np.ascontiguousarray(routed, np.uint8)
    keys = np.empty(max(k, 1), np.uint64)
    est = np.empty(max(k, 1), np.int32)
    n = _load().or_topk_unrouted(_ptr(C), p.rows, p.log2_width, _ptr(p.seeds), p.G, _ptr(routed),
                                 R, k, _ptr(keys), _ptr(est))
    allk = np.concatenate([keys[:n], np.asarray(table_keys, np.uint64)])
    alle = np.concatenate([est[:n], np.asarray(table_counts, np.int32)])
    order = sorted(range(allk.size), key=lambda i: (-int(alle[i]), int(allk[i])))[:k]
    return allk[order], alle[order]


def learned_topk_hier(C2, p, C1, q, F: int, c_mult: int, routed, R: int, table_keys,
                      table_counts, k: int, nthreads: int = 1):
    """Hierarchical query of a learned sketch (super sketch C1 of every kept
    particle, fine sketch C2 of the unrouted ones) merged with the exact counts."""
    routed = np.ascontiguousarray(routed, np.uint8)
    keys = np.empty(max(k, 1), np.uint64)
    est = np.empty(max(k, 1), np.int32)
    n = _load().or_topk_hier_unrouted(_ptr(C2), p.rows, p.log2_width, _ptr(p.seeds), _ptr(C1),
                                      q.rows, q.log2_width, _ptr(q.seeds), p.G, F, k, c_mult,
                                      _ptr(routed), R, _ptr(keys), _ptr(est), nthreads)
    allk = np.concatenate([keys[:n], np.asarray(table_keys, np.uint64)])
    alle = np.concatenate([est[:n], np.asarray(table_counts, np.int32)])
    order = sorted(range(allk.size), key=lambda i: (-int(alle[i]), int(allk[i])))[:k]
    return allk[order], alle[order]
