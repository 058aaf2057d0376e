"""Write the oracle's exhaustive top-k of the 10^9-particle benchmark box.

Calls only `synth` (the seeded input) and `oracle` (the CPU restatement of the
method): no value here comes from the CUDA library.  For each sample rate it
runs the oracle's stream update (Algorithm 1, "Processing the stream") over all
10^9 particles of the 500 Mpc/h box (seed 1) into a 5 x 2^24 int32 Count Sketch
(hash seed 1, sample seed 2), then the full search of Algorithm 1 ("Querying
the data structure", CSFS): the estimate of every one of the 5000^3 cells, the
10^4 best kept by (estimate desc, key asc).  The output file holds the ranked
(key, estimate) list and SHA-256 digests of the particle bytes and of the
counters, so a test can tell a different input from a different update.

Usage (about an hour per rate on 8 host cores; 14 GB of host memory):

    python tests/golden/make_fullsize_topk.py --rate 1.0 --rate 0.1
"""
from __future__ import annotations

import argparse
import hashlib
import os
import sys
import time

import numpy as np

_ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

K = 10 ** 4
PARAMS = dict(rows=5, log2_width=24, box=500.0, cell=0.1, hash_seed=1, sample_seed=2)


def golden_path(rate: float) -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)),
                        f"halo_box_1e9_rate{rate:g}_top{K}.txt")


def sha256_of(a: np.ndarray) -> str:
    h = hashlib.sha256()
    flat = a.reshape(-1).view(np.uint8)
    step = 1 << 28
    for i in range(0, flat.size, step):
        h.update(flat[i:i + step])
    return h.hexdigest()


def read_golden(path: str):
    """(meta dict, keys uint64, estimates int32) of a file this script wrote."""
    meta, keys, est = {}, [], []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line:
                continue
            if line.startswith("#"):
                body = line[1:].strip()
                if ":" in body and not body.startswith(" "):
                    name, _, val = body.partition(":")
                    if name and " " not in name:
                        meta[name] = val.strip()
                continue
            a, b = line.split()
            keys.append(int(a))
            est.append(int(b))
    return meta, np.array(keys, np.uint64), np.array(est, np.int32)


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--rate", type=float, action="append", required=True)
    ap.add_argument("--threads", type=int, default=oracle.default_threads())
    args = ap.parse_args()

    spec = synth.scale_box(1)
    t0 = time.time()
    xyz = synth.HaloBox(spec).generate(0, spec.n)
    xyz_sha = sha256_of(xyz)
    print(f"generated {spec.n} particles in {time.time() - t0:.0f} s, sha256 {xyz_sha}",
          flush=True)
    p = oracle.Params(**PARAMS)
    for rate in args.rate:
        t0 = time.time()
        C = oracle.sketch_update(oracle.new_counters(p), p, xyz, rate=rate, nthreads=args.threads)
        c_sha = sha256_of(C)
        t1 = time.time()
        print(f"rate {rate:g}: update {t1 - t0:.0f} s, counters sha256 {c_sha}", flush=True)
        keys, est = oracle.topk_full(C, p, K, nthreads=args.threads)
        t2 = time.time()
        print(f"rate {rate:g}: full search of {p.n_cells} cells {t2 - t1:.0f} s", flush=True)
        path = golden_path(rate)
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            f.write("# Oracle top-k of the 10^9-particle, 500 Mpc/h halo box (synth.scale_box(1)),\n")
            f.write("# written by tests/golden/make_fullsize_topk.py (oracle and synth only).\n")
            f.write("# Algorithm 1 of arXiv:1711.00975: stream update, then the full search\n")
            f.write("# (CSFS) over every cell of the 5000^3 mesh; ranked by estimate desc, key asc.\n")
            f.write(f"# rows: {p.rows}\n# log2_width: {p.log2_width}\n# box: {p.box:g}\n")
            f.write(f"# cell: {p.cell:g}\n# hash_seed: {p.hash_seed}\n")
            f.write(f"# sample_seed: {p.sample_seed}\n# rate: {rate:g}\n# k: {K}\n")
            f.write(f"# particles: {spec.n}\n# particles_sha256: {xyz_sha}\n")
            f.write(f"# counters_sha256: {c_sha}\n")
            f.write("# columns: key estimate\n")
            for a, b in zip(keys.tolist(), est.tolist()):
                f.write(f"{a} {b}\n")
        os.replace(tmp, path)
        print(f"wrote {path}", flush=True)


if __name__ == "__main__":
    main()
