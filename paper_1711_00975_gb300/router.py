"""Training of the learned router's MLP (an addition to arXiv:1711.00975,
which finds heavy cells with the Count Sketch of Sec. 2.2 alone).

Examples come from training boxes held in device memory: the library's
sample pass gives each coarse cell with a sample its 27 features, and the
library's exact counter (the exact algorithm of Sec. 4.2) gives the labels.  A
coarse cell is positive iff it contains a fine cell whose exact count is at
least the k_label-th largest exact count of its box.  The loss is
class-weighted binary cross-entropy (each class carries half the total weight)
and the optimiser Adam, both in the library's kernels; this module only
assembles examples and feeds mini-batches.
"""
from __future__ import annotations

import numpy as np

from . import halosketch as hs


def box_examples(xyz, n: int, box: float, cell: float, mlp: hs.MLP, coarse_factor: int = 10,
                 feature_seed: int = 64, feature_rate: float = 1.0 / 64, k_label: int = 80,
                 log2_slots: int = 24, stream=None, learned: hs.Learned | None = None,
                 exact: hs.Exact | None = None):
    """(features uint16 [m, 27], labels float32 [m], coarse keys [m]) of one box (device xyz).

    `learned` / `exact` may be passed in to reuse their device memory across
    boxes of the same geometry (they are reset here)."""
    own_l = learned is None
    own_e = exact is None
    L = learned if learned is not None else hs.Learned(
        1, 16, box, cell, coarse_factor=coarse_factor, table_log2=12, feature_seed=feature_seed,
        feature_rate=feature_rate, stream=stream)
    E = exact if exact is not None else hs.Exact(box, cell, log2_slots, stream)
    try:
        L.prepare(xyz, mlp, n)
        ckeys, _ = L.logits()
        feats = L.features()
        if not own_e:
            E.reset()
        E.add(xyz, n)
        # every cell with a count >= the k_label-th largest (ties included)
        want = k_label
        while True:
            keys, counts = E.topk(want)
            if counts.size < want or counts[-1] < counts[min(k_label, counts.size) - 1]:
                break
            want *= 2
    finally:
        if own_l:
            L.close()
        if own_e:
            E.close()
    # examples in coarse-key order: the library lists coarse cells in the
    # order its threads reach them, and training must not depend on that
    order = np.argsort(ckeys, kind="stable")
    ckeys, feats = ckeys[order], feats[order]
    if counts.size == 0:
        return feats, np.zeros(len(ckeys), np.float32), ckeys
    fk = counts[min(k_label, counts.size) - 1]
    heavy = keys[counts >= fk].astype(np.int64)
    G = int(round(box / cell))
    R = coarse_factor
    Gc = G // R
    cx, cy, cz = heavy % G, (heavy // G) % G, heavy // (G * G)
    hot = np.unique(cx // R + Gc * (cy // R + Gc * (cz // R)))
    y = np.isin(ckeys.astype(np.int64), hot).astype(np.float32)
    return feats, y, ckeys


def class_weights(y: np.ndarray) -> np.ndarray:
    """Each class carries half of the total weight len(y)."""
    npos = float(y.sum())
    nneg = float(y.size - npos)
    w = np.where(y > 0, y.size / (2 * max(npos, 1.0)), y.size / (2 * max(nneg, 1.0)))
    return w.astype(np.float32)


def train(mlp: hs.MLP, feats: np.ndarray, y: np.ndarray, epochs: int = 4, batch: int = 65536,
          lr: float = 1e-3, seed: int = 0, device: str = "cuda"):
    """Adam on shuffled mini-batches; returns the mean loss of each epoch."""
    import torch

    w = class_weights(y)
    rng = np.random.default_rng(seed)
    perm = rng.permutation(y.size)
    f_d = torch.from_numpy(np.ascontiguousarray(feats[perm])).to(device)
    y_d = torch.from_numpy(y[perm]).to(device)
    w_d = torch.from_numpy(w[perm]).to(device)
    out = []
    for _ in range(epochs):
        tot = 0.0
        steps = 0
        for b0 in range(0, y.size, batch):
            b1 = min(y.size, b0 + batch)
            tot += mlp.train_step(f_d[b0:b1], y_d[b0:b1], w_d[b0:b1], lr)
            steps += 1
        out.append(tot / max(steps, 1))
    return out
