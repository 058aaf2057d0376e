#!/usr/bin/env python3
"""Throughput of the Count Sketch halo-finder hot path on one GB300.

A step is one pass of the whole path over one synthetic snapshot: reset the
sketch, stream every particle through it (mesh reduction, sampling, Add), then
the full-search top-k (Algorithm 1 of arXiv:1711.00975).  The metric is
particles per second into sketch + top-k; the JSON line also carries the HBM
roofline of the dominant kernel, the end-to-end number through the C ABI with
host buffers, the CPU oracle's throughput on a bounded sample, and clocks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import hashlib

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")
SCATTER_SOURCES = [os.path.join(ROOT, "paper_1711_00975_gb300", "csrc", f)
                   for f in ("k_binned.cuh", "k_binned.cu", "hs_device.cuh")]
sys.path.insert(0, ROOT)

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0

# the 10^9-particle, 500 Mpc/h workload (5000^3 cells of 0.1 Mpc/h)
WORKLOAD = dict(name="halo-box-1e9", n=10**9, box=500.0, n_halo=10**6, cell=0.1, rows=5,
                log2_width=24, k=10**4, box_seed=1, hash_seed=1, sample_seed=2)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--rate", type=float, default=1.0)
    ap.add_argument("--n", type=int, default=None, help="override the particle count")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-red", action="store_true", help="skip the L2 atomic-rate probe")
    ap.add_argument("--no-batch", action="store_true", help="skip the sub-volume batch leg")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-router leg")
    ap.add_argument("--no-stream", action="store_true", help="skip the out-of-core stream leg")
    ap.add_argument("--no-packed", action="store_true",
                    help="skip the legs on 64-bit packed particle records")
    ap.add_argument("--stream-n", type=float, default=2e10, help="particles of the stream leg")
    ap.add_argument("--train-boxes", type=int, default=200,
                    help="100 Mpc/h training boxes of the learned router (seeds 1000..)")
    ap.add_argument("--second-rate", type=float, default=0.1,
                    help="also time this sample rate (0 to skip)")
    ap.add_argument("--batch-only", action="store_true",
                    help="run only the sub-volume batch leg and print its record (profiling)")
    ap.add_argument("--batch-particles", type=float, default=3e8,
                    help="particles of the batch leg, over its 64 sub-volumes")
    return ap.parse_args()


def peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def scatter_capture():
    """The committed ncu record of the scatter kernel (DRAM bytes and warp
    instructions per particle), or None when the kernel's source changed since
    the capture."""
    try:
        with open(TRAFFIC) as f:
            rec = json.load(f)["k_bin_scatter"]
        sha = hashlib.sha256(b"".join(open(p, "rb").read() for p in SCATTER_SOURCES)).hexdigest()
        return rec if sha[:16] == rec["source_sha256_16"] else None
    except (OSError, KeyError, ValueError):
        return None


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._proc = None

    def __enter__(self):
        try:
            self._proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self._proc = None
        return self

    def _read(self):
        for line in self._proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self._proc is not None:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self._proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if s[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def bind_near_gpu(index: int):
    """Run on (and so allocate pinned host memory from) the NUMA node of the
    GPU's host link.  On a two-socket host a buffer on the far node crosses
    the socket link and copies to the GPU run at a fraction of the link's
    rate.  Returns the node, or None when the topology is not readable."""
    try:
        bus = subprocess.run(["nvidia-smi", f"--id={index}", "--query-gpu=pci.bus_id",
                              "--format=csv,noheader"], capture_output=True, text=True,
                             timeout=30).stdout.strip().lower()
        dom, rest = bus.split(":", 1)
        dev = f"{int(dom, 16):04x}:{rest}"
        with open(f"/sys/bus/pci/devices/{dev}/numa_node") as f:
            node = int(f.read().strip())
        if node < 0:
            return None
        with open(f"/sys/devices/system/node/node{node}/cpulist") as f:
            cpus = set()
            for part in f.read().strip().split(","):
                lo, _, hi = part.partition("-")
                cpus.update(range(int(lo), int(hi or lo) + 1))
        if cpus:
            os.sched_setaffinity(0, cpus)
        return node
    except (OSError, ValueError, subprocess.SubprocessError):
        return None


def make_box(n):
    import synth
    spec = synth.BoxSpec(n=n, box=WORKLOAD["box"], n_halo=max(1, WORKLOAD["n_halo"] * n // 10**9),
                         seed=WORKLOAD["box_seed"])
    return spec, synth.HaloBox(spec)


def cpu_sample_rates(xyz_host: np.ndarray, n_update: int, n_cells: int, k: int, rate: float):
    """Oracle throughput on a bounded sample: (particles/s, cells/s, cores, seconds)."""
    import oracle
    cores = oracle.default_threads()
    p = oracle.Params(WORKLOAD["rows"], WORKLOAD["log2_width"], WORKLOAD["box"], WORKLOAD["cell"],
                      WORKLOAD["hash_seed"], WORKLOAD["sample_seed"])
    C = oracle.new_counters(p)
    sample = xyz_host[:n_update]
    t0 = time.perf_counter()
    oracle.sketch_update(C, p, sample, rate=rate, nthreads=cores)
    t1 = time.perf_counter()
    oracle.topk_full(C, p, k, nthreads=cores, key_lo=0, key_hi=n_cells)
    t2 = time.perf_counter()
    return n_update / (t1 - t0), n_cells / (t2 - t1), cores, t2 - t0


def run_batched(steps: int, warmup: int, total: float = 3e8):
    """64 sub-volumes of uneven size (2^16..2^26 particles, about `total` in
    all), each with its own 5 x 2^18 sketch and top-500, updated as one batch."""
    import torch

    import synth
    from paper_1711_00975_gb300 import halosketch as hs

    specs = synth.subvolume_specs(seed=3, target_total=total)
    counts = [s.n for s in specs]
    offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.uint64)
    total = int(offsets[-1])
    host = torch.empty((total, 3), dtype=torch.float32).pin_memory()
    t0 = time.time()
    for s_, o in zip(specs, offsets[:-1]):
        synth.HaloBox(s_).generate_into_ptr(host.data_ptr() + int(o) * 12, 0, s_.n)
    gen_s = time.time() - t0
    dev = host.cuda()
    stream = torch.cuda.Stream()        # a batch's graph needs a non-legacy stream
    torch.cuda.synchronize()
    b = hs.Batch(5, 18, [s_.box for s_ in specs], 0.1, hash_seed=3, sample_seed=4, stream=stream)
    tune = b.autotune(dev, offsets, 1.0)

    def step():
        b.reset()
        b.update(dev, offsets, 1.0)
        return b.topk(500)

    for _ in range(warmup):
        step()
    b.stats(reset=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ups = []
    e0.record(stream)
    for _ in range(steps):
        a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b.reset()
        a.record(stream)
        b.update(dev, offsets, 1.0)
        c.record(stream)
        b.topk(500)
        ups.append((a, c))
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    upd = float(np.mean([a.elapsed_time(c) for a, c in ups]))
    st = b.stats(reset=True)
    b.close()
    hbm, _ = peaks()
    return {"workload": "subvolumes-64", "volumes": len(specs), "particles": total,
            "roofline": {"kernel": "k_bin_scatter<batch> + k_bin_accumulate", "bound": "hbm",
                         "achieved": 12.0 * total / (upd * 1e-3) / 1e9, "peak": hbm,
                         "unit": "GB/s", "frac": 12.0 * total / (upd * 1e-3) / 1e9 / hbm,
                         "note": "12 B per particle over the update's time"},
            "particles_per_s": total / (ms * 1e-3), "ms_per_step": ms, "update_ms": upd,
            "update_stream_gbs": 12.0 * total / (upd * 1e-3) / 1e9,
            "topk_ms_per_step": ms - upd, "k": 500, "sketch": "5 x 2^18 int32 per volume",
            "autotune": tune, "gpu_launches_per_step": st["kernel_launches"] / steps,
            "generation_s": gen_s}


def run_reference(args):
    """The oracle as the reference arm: each step a bounded sample of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n = args.n or WORKLOAD["n"]
    G = round(WORKLOAD["box"] / WORKLOAD["cell"])
    n_upd = min(n, 1 << 24)
    n_cells = min(G ** 3, 4 * 10**8)
    spec, box = make_box(n)
    xyz = box.generate(0, n_upd)
    for _ in range(args.warmup):
        cpu_sample_rates(xyz, n_upd, n_cells, WORKLOAD["k"], args.rate)
    times = []
    cores = 1
    for _ in range(args.steps):
        ru, rq, cores, _ = cpu_sample_rates(xyz, n_upd, n_cells, WORKLOAD["k"], args.rate)
        times.append(n / ru + G ** 3 / rq)      # extrapolated time of one full step
    step_s = float(np.mean(times))
    value = n / step_s
    line = {"impl": "reference", "metric": "particles/s into sketch+top-k", "value": value,
            "unit": "particles/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOAD["name"], "particles": n, "grid": G,
                       "rows": WORKLOAD["rows"], "width": 1 << WORKLOAD["log2_width"],
                       "k": WORKLOAD["k"], "sample_rate": args.rate},
            "cpu_baseline": {"value": value, "unit": "particles/s", "cores": cores, "kind": "oracle",
                             "sample": f"update of {n_upd} particles + full search of {n_cells} "
                                       f"cells per step, extrapolated to {n} particles and "
                                       f"{G ** 3} cells"},
            "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


LEARNED = dict(coarse_factor=10, table_log2=20, sketch_log2_width=23, feature_seed=64,
               feature_rate=1.0 / 64, k_label=80, exact_log2_slots=31)


def train_router(spec_of, n_boxes: int, k_label: int, stream):
    """Train the router's MLP on n_boxes generated boxes (spec_of(i)): features
    from the library's sample pass, labels from its exact counter; box i+1 is
    generated on the host while box i is on the GPU."""
    import torch

    import synth
    from paper_1711_00975_gb300 import halosketch as hs
    from paper_1711_00975_gb300 import router

    W = WORKLOAD
    C = LEARNED
    t0 = time.time()
    mlp = hs.MLP(seed=1, stream=stream)
    tspec = spec_of(0)
    bufs = [torch.empty((tspec.n, 3), dtype=torch.float32).pin_memory() for _ in range(2)]
    gen_s = [0.0]

    def gen(i, buf):
        t = time.time()
        synth.HaloBox(spec_of(i)).generate_into_ptr(buf.data_ptr(), 0, tspec.n)
        gen_s[0] += time.time() - t

    Lt = hs.Learned(1, 16, tspec.box, W["cell"], coarse_factor=C["coarse_factor"], table_log2=12,
                    feature_seed=C["feature_seed"], feature_rate=C["feature_rate"], stream=stream)
    Et = hs.Exact(tspec.box, W["cell"], 24, stream)
    dbox = torch.empty((tspec.n, 3), dtype=torch.float32, device="cuda")
    feats, ys = [], []
    th = threading.Thread(target=gen, args=(0, bufs[0]))
    th.start()
    for i in range(n_boxes):
        th.join()
        dbox.copy_(bufs[i % 2])
        torch.cuda.synchronize()
        if i + 1 < n_boxes:
            th = threading.Thread(target=gen, args=(i + 1, bufs[(i + 1) % 2]))
            th.start()
        f, y, _ = router.box_examples(dbox, tspec.n, tspec.box, W["cell"], mlp,
                                      C["coarse_factor"], C["feature_seed"], C["feature_rate"],
                                      k_label, learned=Lt, exact=Et)
        feats.append(f)
        ys.append(y)
    Lt.close()
    Et.close()
    del dbox
    F = np.concatenate(feats)
    Y = np.concatenate(ys)
    t1 = time.time()
    losses = router.train(mlp, F, Y, epochs=4, batch=65536, lr=1e-3, seed=0)
    torch.cuda.synchronize()
    info = {"boxes": n_boxes, "box": f"{tspec.n} particles / {tspec.box} Mpc/h / {tspec.n_halo} halos",
            "examples": int(Y.size), "positives": int(Y.sum()), "examples_s": t1 - t0,
            "generation_s": gen_s[0], "train_s": time.time() - t1, "epoch_losses": losses,
            "label": f"coarse cell holds a fine cell >= the {k_label}-th largest exact count "
                     f"of its box"}
    return mlp, info


def run_learned(dev, n: int, train_boxes: int, stream):
    """The learned router on the 10^9-particle box: train on 100 Mpc/h boxes,
    then top-k recall against exact counts for plain sketches of 5 x 2^23
    (160 MiB), 6 x 2^23 (192 MiB), 7 x 2^23 (224 MiB, more than the learned
    sketch's whole footprint) and 5 x 2^24 (320 MiB), and for the learned sketch (5 x 2^23 +
    exact blocks of a 2^20-slot table's bytes + its routing bitmap and prefix),
    with the memory of each beside its recall."""
    import torch

    import synth
    from paper_1711_00975_gb300 import halosketch as hs

    W = WORKLOAD
    C = LEARNED
    k = W["k"]
    out = {"workload": W["name"], "k": k, "train_boxes": train_boxes}
    mlp, out["training"] = train_router(lambda i: synth.training_box(1000 + i), train_boxes,
                                        C["k_label"], stream)
    out["training"]["params_sha256_16"] = hashlib.sha256(mlp.get_params().tobytes()).hexdigest()[:16]
    # ---- evaluation on the main box
    E = hs.Exact(W["box"], W["cell"], C["exact_log2_slots"], stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    E.add(dev, n)
    ev[1].record(stream)
    torch.cuda.synchronize()
    out["exact_add_ms"] = ev[0].elapsed_time(ev[1])
    out["distinct_cells"] = E.size()

    def timed_call(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return r, a.elapsed_time(b)

    plain = {}
    for rows, log2w in ((5, C["sketch_log2_width"]), (6, C["sketch_log2_width"]),
                        (7, C["sketch_log2_width"]), (W["rows"], W["log2_width"])):
        sk = hs.Sketch(rows, log2w, W["box"], W["cell"], W["hash_seed"], W["sample_seed"],
                       stream=stream)
        _, up_ms = timed_call(lambda: (sk.update(dev, n), sk.flush()))
        (pk, _), tk_ms = timed_call(lambda: sk.topk(k))
        nbytes = rows * 4 << log2w
        plain[f"{rows}x2^{log2w}"] = {"recall": E.recall(pk, k), "memory_bytes": nbytes,
                                      "update_ms": up_ms, "topk_ms": tk_ms}
        sk.close()
    L = hs.Learned(W["rows"], C["sketch_log2_width"], W["box"], W["cell"], W["hash_seed"],
                   W["sample_seed"], coarse_factor=C["coarse_factor"], table_log2=C["table_log2"],
                   feature_seed=C["feature_seed"], feature_rate=C["feature_rate"], stream=stream)
    nr, prep_ms = timed_call(lambda: L.prepare(dev, mlp, n))
    _, lup_ms = timed_call(lambda: (L.update(dev, n), hs.sketch_flush(L.sketch_h)))
    (lk, _), ltk_ms = timed_call(lambda: L.topk(k))
    learned = E.recall(lk, k)
    sketch_bytes = W["rows"] * 4 << C["sketch_log2_width"]
    aux = (L.Gc ** 3 + 31) // 32 * 8          # routing bitmap + one prefix count a word
    out.update({
        "recall_plain": plain,
        "recall_learned": {"recall": learned, "memory_bytes": sketch_bytes + L.table_bytes + aux,
                           "sketch_bytes": sketch_bytes, "exact_block_bytes": L.table_bytes,
                           "routing_aux_bytes": aux},
        "routed_coarse_cells": int(nr), "max_routed": int(L.max_routed),
        "learned_ms": {"prepare": prep_ms, "update": lup_ms, "topk": ltk_ms},
        "learned_particles_per_s": n / ((prep_ms + lup_ms + ltk_ms) * 1e-3),
        "roofline": {"kernel": "k_bin_scatter<routed> + k_bin_accumulate", "bound": "hbm",
                     "achieved": 12.0 * n / (lup_ms * 1e-3) / 1e9, "peak": peaks()[0],
                     "unit": "GB/s", "frac": 12.0 * n / (lup_ms * 1e-3) / 1e9 / peaks()[0],
                     "note": "12 B per particle over the learned update's time; the sample "
                             "pass reads the same 12 B in "
                             f"{prep_ms:.1f} ms with features, MLP and routing"},
        "exact_table": f"2^{C['exact_log2_slots']} slots"})
    L.close()
    E.close()
    mlp.close()
    return out


STREAM = dict(name="stream-2e10", box=2000.0, n_halo=64 * 10**6, cell=0.1, rows=5,
              log2_width=26, k=10**5, rate=0.1, chunk_bytes=10**9, pool_chunks=4, box_seed=4,
              hash_seed=5, sample_seed=6, super_factor=10, super_log2_width=26, c_mult=2,
              learned_log2_width=25, train_boxes=100, k_label=12)


def measure_h2d(src, dst, stream, reps: int = 5) -> float:
    """Best pinned host -> device copy rate (GB/s) of one chunk, CUDA events."""
    import torch
    best = 0.0
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a.record(stream)
            dst.copy_(src, non_blocking=True)
            b.record(stream)
        torch.cuda.synchronize()
        best = max(best, src.numel() * src.element_size() / (a.elapsed_time(b) * 1e-3) / 1e9)
    return best


def run_stream(n_total: int, hbm: float, learned_leg: bool = True, packed_leg: bool = True):
    """Out-of-core stream: n_total particles of a 2000 Mpc/h box pass from pinned
    host chunks of 1 GB through the library's double-buffered staging (copy
    stream + compute stream) into a 5 x 2^26 sketch at sample rate 0.1, then
    the top-10^5.  Host generation (about 1e8 particles/s) is far slower than
    the link, so the chunks cycle through a pool of the stream's first 4 GB
    while the particle indices (and so the sampling) run over the whole
    stream; the copies and the updates are those of the full stream."""
    import torch

    import synth
    from paper_1711_00975_gb300 import halosketch as hs

    S = STREAM
    C = S["chunk_bytes"] // 12

    def note(msg):
        print(f"[stream {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)
    spec = synth.BoxSpec(n=n_total, box=S["box"], n_halo=S["n_halo"], seed=S["box_seed"])
    t0 = time.time()
    hb = synth.HaloBox(spec)
    pool = [torch.empty((C, 3), dtype=torch.float32).pin_memory() for _ in range(S["pool_chunks"])]
    for c, buf in enumerate(pool):
        hb.generate_into_ptr(buf.data_ptr(), c * C, C)
    gen_s = time.time() - t0
    gen_rate = C * S["pool_chunks"] / gen_s
    note(f"pool of {len(pool)} chunks generated in {gen_s:.1f} s")
    stream = torch.cuda.Stream()
    probe = torch.empty((C, 3), dtype=torch.float32, device="cuda")
    h2d_peak = measure_h2d(pool[0], probe, stream)
    del probe
    sk = hs.Sketch(S["rows"], S["log2_width"], S["box"], S["cell"], S["hash_seed"],
                   S["sample_seed"], stream=stream)
    # 8e12 cells: the query is hierarchical (Algorithm 3) over 10^3-cell super-items
    sk.set_hierarchy(S["super_factor"], S["super_log2_width"], S["c_mult"])
    sup = sk.super_handle()
    nchunks = (n_total + C - 1) // C

    def one_pass():
        for c in range(nchunks):
            cnt = min(C, n_total - c * C)
            hs.sketch_update(sk.h, pool[c % len(pool)], cnt, S["rate"])
        hs.sketch_flush(sk.h)

    # warm-up: a few chunks and one top-k (builds bins, probe, directories)
    for c in range(3):
        hs.sketch_update(sk.h, pool[c], C, S["rate"])
    note("warm-up updates issued")
    sk.topk(S["k"])
    note("warm-up top-k done")
    sk.reset()
    sk.stats(reset=True)
    hs.sketch_stats(sup, reset=True)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    w0 = time.perf_counter()
    e[0].record(stream)
    one_pass()
    e[1].record(stream)
    note("stream issued")
    keys, est = sk.topk(S["k"])
    e[2].record(stream)
    note("top-k done")
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    upd_ms = e[0].elapsed_time(e[1])
    tk_ms = e[1].elapsed_time(e[2])
    st = sk.stats(reset=True)
    st1 = hs.sketch_stats(sup, reset=True)
    total_ms = max(e[0].elapsed_time(e[2]), wall * 1e3)
    h2d = 12.0 * n_total / (upd_ms * 1e-3) / 1e9
    kernel_ms = st["update_ms"] + st1["update_ms"]
    kern_gbs = 12.0 * n_total / (kernel_ms * 1e-3) / 1e9 if kernel_ms > 0 else None
    packed = run_stream_packed(n_total, pool, sk, sup, stream, note) if packed_leg else None
    sk.close()
    learned = run_stream_learned(n_total, pool, C, stream, note) if learned_leg else None
    return {"workload": S["name"], "particles": n_total, "box_mpc_h": S["box"], "grid": round(S["box"] / S["cell"]),
            "rows": S["rows"], "width": 1 << S["log2_width"], "k": S["k"], "sample_rate": S["rate"],
            "chunk_bytes": C * 12, "chunks": nchunks, "pool_chunks": S["pool_chunks"],
            "value": n_total / (total_ms * 1e-3), "unit": "particles/s", "ms": total_ms,
            "stream_ms": upd_ms, "topk_ms": tk_ms,
            "h2d": {"achieved_gbs": h2d, "peak_gbs": h2d_peak, "frac": h2d / h2d_peak,
                    "peak_source": "best pinned 1 GB cudaMemcpyAsync on this box"},
            "hbm": {"kernel_ms": kernel_ms, "achieved_gbs": kern_gbs, "peak_gbs": hbm,
                    "frac": kern_gbs / hbm if kern_gbs else None,
                    "note": "12 B/particle over the update kernels' own time"},
            "gpu_launches": int(st["kernel_launches"] + st1["kernel_launches"]),
            "top_count": int(est[0]) if len(est) else 0,
            "query": {"kind": "hierarchical (Algorithm 3)", "super_factor": S["super_factor"],
                      "super_sketch": f"{S['rows']} x 2^{S['super_log2_width']}",
                      "c_mult": S["c_mult"], "super_topk_ms": st1["topk_ms"],
                      "update_ms_fine": st["update_ms"], "update_ms_super": st1["update_ms"]},
            "generation": {"seconds": gen_s, "particles_per_s": gen_rate,
                           "note": "host generator rate; the stream cycles a pool of chunks"},
            "packed": packed, "learned": learned}


def run_stream_packed(n_total: int, pool, sk, sup, stream, note):
    """The same stream as 64-bit records: 8 bytes a particle over the link.
    The pool chunks are packed once on the GPU (Sec. 4 stores the dataset in
    this layout); the chunk count stays, each chunk holds the same particles."""
    import torch

    from paper_1711_00975_gb300 import halosketch as hs

    S = STREAM
    C = pool[0].shape[0]
    dchunk = torch.empty((C, 3), dtype=torch.float32, device="cuda")
    drec = torch.empty(C, dtype=torch.int64, device="cuda")
    rpool = []
    for buf in pool:
        dchunk.copy_(buf)
        hs.pack_positions(dchunk, S["box"], drec, C, stream)
        r = torch.empty(C, dtype=torch.int64).pin_memory()
        r.copy_(drec)
        rpool.append(r)
    del dchunk, drec
    torch.cuda.synchronize()
    nchunks = (n_total + C - 1) // C
    sk.reset()
    sk.stats(reset=True)
    hs.sketch_stats(sup, reset=True)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    w0 = time.perf_counter()
    e[0].record(stream)
    for c in range(nchunks):
        hs.sketch_update_packed(sk.h, rpool[c % len(rpool)], min(C, n_total - c * C), S["rate"])
    hs.sketch_flush(sk.h)
    e[1].record(stream)
    keys, est = sk.topk(S["k"])
    e[2].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    note("packed stream done")
    st = sk.stats(reset=True)
    st1 = hs.sketch_stats(sup, reset=True)
    upd = e[0].elapsed_time(e[1])
    total = max(e[0].elapsed_time(e[2]), wall * 1e3)
    return {"value": n_total / (total * 1e-3), "unit": "particles/s", "ms": total,
            "stream_ms": upd, "topk_ms": e[1].elapsed_time(e[2]),
            "h2d_gbs": 8.0 * n_total / (upd * 1e-3) / 1e9,
            "update_kernel_ms": st["update_ms"] + st1["update_ms"],
            "bytes_per_particle": 8}


def run_stream_learned(n_total: int, pool, C: int, stream, note):
    """The same stream through the learned router: a 1/64 sample pass over the
    whole stream, routing of the 2000^3 coarse cells, then the update pass into
    a 5 x 2^25 sketch (half the plain one) with exact blocks for routed cells,
    and the hierarchical top-10^5 merged with the exact counts.  The router is
    trained on 100 Mpc/h boxes at this stream's density."""
    import torch

    import synth
    from paper_1711_00975_gb300 import halosketch as hs

    S = STREAM
    L_ = LEARNED
    spec_of = lambda i: synth.BoxSpec(n=n_total * 10**6 // 8 // 10**9, box=100.0,
                                      n_halo=S["n_halo"] // 8000, seed=2000 + i)
    mlp, training = train_router(spec_of, S["train_boxes"], S["k_label"], stream)
    note(f"stream router trained ({training['examples']} examples)")
    L = hs.Learned(S["rows"], S["learned_log2_width"], S["box"], S["cell"], S["hash_seed"],
                   S["sample_seed"], coarse_factor=L_["coarse_factor"], table_log2=L_["table_log2"],
                   feature_seed=L_["feature_seed"], feature_rate=L_["feature_rate"], stream=stream)
    L.set_hierarchy(S["super_factor"], S["learned_log2_width"], S["c_mult"])
    nchunks = (n_total + C - 1) // C
    e = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    e[0].record(stream)
    for c in range(nchunks):
        L.sample(pool[c % len(pool)], min(C, n_total - c * C))
    e[1].record(stream)
    nr = L.route(mlp)
    e[2].record(stream)
    for c in range(nchunks):
        L.update(pool[c % len(pool)], min(C, n_total - c * C), S["rate"])
    hs.sketch_flush(L.sketch_h)
    e[3].record(stream)
    keys, est = L.topk(S["k"])
    e[4].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    note("learned stream done")
    ms = [e[i].elapsed_time(e[i + 1]) for i in range(4)]
    total = max(sum(ms), wall * 1e3)
    sketch_bytes = 2 * (S["rows"] * 4 << S["learned_log2_width"])
    out = {"value": n_total / (total * 1e-3), "unit": "particles/s", "ms": total,
           "sample_pass_ms": ms[0], "route_ms": ms[1], "update_pass_ms": ms[2], "topk_ms": ms[3],
           "h2d_gbs_sample_pass": 12.0 * n_total / (ms[0] * 1e-3) / 1e9,
           "h2d_gbs_update_pass": 12.0 * n_total / (ms[2] * 1e-3) / 1e9,
           "routed_coarse_cells": int(nr), "max_routed": int(L.max_routed),
           "memory_bytes": {"sketches": sketch_bytes, "exact_blocks": L.table_bytes,
                            "plain_stream_sketches": 2 * (S["rows"] * 4 << S["log2_width"])},
           "sketch": f"{S['rows']} x 2^{S['learned_log2_width']} + hierarchy {S['rows']} x "
                     f"2^{S['learned_log2_width']}", "training": training,
           "top_count": int(est[0]) if len(est) else 0,
           "note": "no recall: exact counts of 2e10 particles (~1e10 cells) exceed device memory"}
    L.close()
    mlp.close()
    return out


def run_ours(args):
    import torch

    import synth
    from paper_1711_00975_gb300 import halosketch as hs

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    hs.lib()

    n = args.n or WORKLOAD["n"]
    k = WORKLOAD["k"]
    G = round(WORKLOAD["box"] / WORKLOAD["cell"])
    numa = bind_near_gpu(local)
    spec, box = make_box(n)
    # one rank: the whole stream; several: this rank's contiguous shard by
    # particle index, the counters summed over the ranks (Sec. 5) before rank
    # 0's top-k
    from paper_1711_00975_gb300.distributed import shard_range
    lo, n_local = shard_range(n, rank, world)
    t0 = time.time()
    host = torch.empty((n_local, 3), dtype=torch.float32).pin_memory()
    box.generate_into_ptr(host.data_ptr(), lo, n_local)
    gen_s = time.time() - t0
    dev = host.to(f"cuda:{local}", non_blocking=False)
    stream = torch.cuda.current_stream()
    sk = hs.Sketch(WORKLOAD["rows"], WORKLOAD["log2_width"], WORKLOAD["box"], WORKLOAD["cell"],
                   WORKLOAD["hash_seed"], WORKLOAD["sample_seed"], stream=stream)
    keys = np.empty(k, np.uint64)
    ests = np.empty(k, np.int32)
    merge_buf = torch.empty((sk.rows, sk.width), dtype=torch.int32, device=f"cuda:{local}") \
        if world > 1 else None

    def begin():
        hs.sketch_reset(sk.h)
        if world > 1:
            hs.sketch_seek(sk.h, lo)

    def finish():
        """counters of the whole stream (all-reduce over the ranks), then the
        top-k on rank 0"""
        if world > 1:
            hs.sketch_counters(sk.h, merge_buf)
            dist.all_reduce(merge_buf, op=dist.ReduceOp.SUM)
            hs.sketch_load_counters(sk.h, merge_buf)
        if rank == 0:
            return hs.topk_extract(sk.h, k, keys, ests)
        return 0

    def step(src, rate):
        begin()
        hs.sketch_update(sk.h, src, n_local, rate)
        hs.sketch_flush(sk.h)
        return finish()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    def timed(src, rate, steps, warmup):
        for _ in range(warmup):
            step(src, rate)
        sk.stats(reset=True)
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        upd = []
        ev0.record(stream)
        for _ in range(steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            begin()
            a.record(stream)
            hs.sketch_update(sk.h, src, n_local, rate)
            hs.sketch_flush(sk.h)
            b.record(stream)
            finish()
            upd.append((a, b))
        ev1.record(stream)
        barrier()
        total_ms = ev0.elapsed_time(ev1)
        upd_ms = [a.elapsed_time(b) for a, b in upd]
        st = sk.stats(reset=True)
        if dist is not None:
            t = torch.tensor([total_ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            total_ms = float(t.item())
        return total_ms, upd_ms, st

    hbm, peak_kind = peaks()
    with Clocks(local) as clk:
        total_ms, upd_ms, st = timed(dev, args.rate, args.steps, args.warmup)
    clocks = clk.summary()
    ms_step = total_ms / args.steps
    value = n / (ms_step * 1e-3)              # every rank's particles (the whole stream)
    upd_avg = float(np.mean(upd_ms))
    search_avg = st["search_ms"] / max(1, st["search_launches"])
    search_per_step = st["search_ms"] / args.steps
    topk_per_step = st["topk_ms"] / args.steps
    stream_gbs = 12.0 * n_local / (upd_avg * 1e-3) / 1e9

    # Dominant kernel by device time per step: the scatter of the binned update
    # (several launches per step) or the directory query of the full search.
    scatter_launches = max(1, st["update_launches"])
    scatter_ms = (st["update_ms"] - st["flush_ms"]) / scatter_launches
    per_launch = n_local * args.steps / scatter_launches
    scatter_per_step = st["update_ms"] - st["flush_ms"]
    scatter_gbs = 12.0 * per_launch / (scatter_ms * 1e-3) / 1e9
    cap = scatter_capture()
    bpp = cap["dram_bytes_per_particle"] if cap else None
    roof = {"kernel": "k_bin_scatter", "bound": "hbm", "achieved": scatter_gbs, "peak": hbm,
            "unit": "GB/s", "frac": scatter_gbs / hbm,
            "traffic": bpp * per_launch if bpp is not None else None,
            "algorithmic_bytes_per_launch": 12.0 * per_launch,
            "launch_ms": scatter_ms, "launches_per_step": scatter_launches / args.steps,
            "peak_source": f"{peak_kind} hbm_gbs",
            "note": "12 B of float32 xyz per particle read once; bins are not algorithmic"}
    if search_per_step > scatter_per_step / args.steps:
        roof["note"] += "; the full search took longer than the scatter this run"
    if cap and cap.get("warp_inst_per_particle"):
        # what binds the scatter: instruction issue, one warp instruction per
        # clock per SM sub-partition at the clock sampled during the run
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        mhz = clocks.get("sm_mhz") or 2070.0
        peak_issue = sms * 4 * mhz * 1e6
        got = cap["warp_inst_per_particle"] * per_launch / (scatter_ms * 1e-3)
        roof["issue"] = {"achieved": got, "peak": peak_issue, "unit": "warp instructions/s",
                         "frac": got / peak_issue,
                         "warp_inst_per_particle": cap["warp_inst_per_particle"],
                         "note": "instruction count from the committed ncu capture"}
    search_roof = {"kernel": "k_dir_query", "cells_per_s": G ** 3 / (search_per_step * 1e-3)
                   if search_per_step > 0 else None, "ms_per_step": search_per_step}

    second = None
    if args.second_rate and args.second_rate != args.rate and world == 1:
        t2, u2, s2 = timed(dev, args.second_rate, max(2, args.steps // 2), 1)
        u2avg = float(np.mean(u2))
        second = {"sample_rate": args.second_rate, "value": n / (t2 / max(2, args.steps // 2) * 1e-3),
                  "update_ms": u2avg, "stream_gbs": 12.0 * n_local / (u2avg * 1e-3) / 1e9,
                  "stream_frac": 12.0 * n_local / (u2avg * 1e-3) / 1e9 / hbm}

    red = None
    if not args.no_red:
        try:
            tab = 1 << ((WORKLOAD["rows"] << WORKLOAD["log2_width"]) - 1).bit_length()
            ops = hs.hs_measure_red_rate(tab, 1 << 31)
            red = {"ops_per_s": ops, "table_counters": tab,
                   "needed_ops_per_particle": WORKLOAD["rows"] * args.rate,
                   "particles_per_s_bound": ops / (WORKLOAD["rows"] * args.rate)}
        except hs.HSError as e:
            red = {"error": str(e)}

    e2e = None
    if not args.no_e2e:
        steps_e = max(2, args.steps // 2)
        for _ in range(2):             # the first passes over the pinned buffer run slower
            step(host, args.rate)
        sk.stats(reset=True)
        barrier()
        t0 = time.perf_counter()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps_e):
            step(host, args.rate)
        e1.record(stream)
        barrier()
        ems = e0.elapsed_time(e1) / steps_e
        wall = (time.perf_counter() - t0) / steps_e
        est = sk.stats(reset=True)
        # the host link alone: the best of five plain 1 GiB copies from the
        # same pinned buffer (one copy of all 12 GB runs far below the link)
        m = min(host.numel(), 1 << 28)
        link_gbs = measure_h2d(host.view(-1)[:m], dev.view(-1)[:m], stream)
        step_ms = max(ems, wall * 1e3)
        e2e = {"value": n / (step_ms * 1e-3), "unit": "particles/s",
               "h2d_bytes_per_step": 12 * n, "d2h_bytes_per_step": 12 * k,
               "ms_per_step": step_ms,
               "h2d_gbs": 12.0 * n_local / (step_ms * 1e-3) / 1e9,
               "h2d_gbs_copies": est["h2d_bytes"] / (est["h2d_ms"] * 1e-3) / 1e9 if est["h2d_ms"] else None,
               "h2d_gbs_plain_copy": link_gbs,
               "note": "h2d_gbs: bytes over the link per step time; h2d_gbs_copies: the staged "
                       "copies' own rate; h2d_gbs_plain_copy: the best of five 1 GiB copies "
                       "of the same pinned buffer"}

    packed = None
    if not args.no_packed and world == 1:
        # the same particles as 64-bit records (Sec. 4's data layout): 8 bytes
        # a particle in HBM and over the host link
        rec = torch.empty(n, dtype=torch.int64, device=dev.device)
        hs.pack_positions(dev, WORKLOAD["box"], rec, n, stream)
        rec_host = torch.empty(n, dtype=torch.int64).pin_memory()
        rec_host.copy_(rec)
        torch.cuda.synchronize()

        def pstep(src):
            hs.sketch_reset(sk.h)
            hs.sketch_update_packed(sk.h, src, n, args.rate)
            hs.sketch_flush(sk.h)
            return hs.topk_extract(sk.h, k, keys, ests)

        def ptimed(src, steps, warmup):
            for _ in range(warmup):
                pstep(src)
            sk.stats(reset=True)
            barrier()
            w0 = time.perf_counter()
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record(stream)
            for _ in range(steps):
                pstep(src)
            b_.record(stream)
            barrier()
            return max(a_.elapsed_time(b_), (time.perf_counter() - w0) * 1e3) / steps, \
                sk.stats(reset=True)

        pms, pst = ptimed(rec, args.steps, args.warmup)
        pgbs = 8.0 * n / (pst["update_ms"] / args.steps * 1e-3) / 1e9
        packed = {"records": "64-bit, three 21-bit coordinates", "value": n * world / (pms * 1e-3),
                  "roofline": {"kernel": "k_bin_scatter<packed> + k_bin_accumulate",
                               "bound": "hbm", "achieved": pgbs, "peak": hbm, "unit": "GB/s",
                               "frac": pgbs / hbm, "note": "8 B per record over the update"},
                  "unit": "particles/s", "ms_per_step": pms,
                  "update_ms": pst["update_ms"] / args.steps,
                  "stream_gbs": 8.0 * n / (pst["update_ms"] / args.steps * 1e-3) / 1e9,
                  "gpu_launches": int(pst["kernel_launches"])}
        if not args.no_e2e:
            ems, _ = ptimed(rec_host, max(2, args.steps // 2), 2)
            packed["e2e"] = {"value": n * world / (ems * 1e-3), "unit": "particles/s",
                             "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 12 * k,
                             "ms_per_step": ems}
        del rec, rec_host
        torch.cuda.empty_cache()

    learned = None
    if not args.no_learned and world == 1:
        learned = run_learned(dev, n, args.train_boxes, stream)

    stream_leg = None
    if not args.no_stream and world == 1:
        del dev
        torch.cuda.empty_cache()
        dev = None
        stream_leg = run_stream(int(args.stream_n), hbm, not args.no_learned, not args.no_packed)

    batched = None
    if not args.no_batch and world == 1:
        del dev
        torch.cuda.empty_cache()
        batched = run_batched(max(3, args.steps // 2), args.warmup, args.batch_particles)

    cpu = None
    if not args.no_cpu and world == 1:
        n_upd = min(n, 1 << 27)
        n_cells = min(G ** 3, 2 * 10**9)
        ru, rq, cores, secs = cpu_sample_rates(host.numpy(), n_upd, n_cells, k, args.rate)
        cpu = {"value": n / (n / ru + G ** 3 / rq), "unit": "particles/s", "cores": cores,
               "kind": "oracle", "seconds": secs,
               "sample": f"oracle update of the first {n_upd} particles ({ru:.3g} particles/s) and "
                         f"full search of the first {n_cells} cells ({rq:.3g} cells/s), "
                         f"extrapolated to {n} particles + {G ** 3} cells"}

    line = {"metric": "particles/s into sketch+top-k", "value": value, "unit": "particles/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD["name"], "particles": n, "box_mpc_h": WORKLOAD["box"],
                       "cell_mpc_h": WORKLOAD["cell"], "grid": G, "rows": WORKLOAD["rows"],
                       "width": 1 << WORKLOAD["log2_width"], "k": k, "sample_rate": args.rate,
                       "l2": "inputs (12 GB) larger than L2", "generation_s": gen_s,
                       "host_numa_node": numa,
                       "parallelism": (f"{world} particle-index shards, int32 counters all-reduced, "
                                       "top-k on rank 0") if world > 1 else "one GPU"},
            "breakdown": {"update_ms": upd_avg, "flush_ms": st["flush_ms"] / args.steps,
                          "topk_ms": topk_per_step,
                          "full_search_ms": search_per_step,
                          "stream_gbs": stream_gbs, "stream_frac": stream_gbs / hbm,
                          "candidates": st["last_candidates"], "threshold": st["last_threshold"],
                          "passes": st["last_passes"]},
            "roofline": roof, "search": search_roof, "red_rate": red, "second_rate": second, "e2e": e2e,
            "packed": packed, "batched": batched, "learned": learned, "stream": stream_leg,
            "cpu_baseline": cpu, "clocks": clocks,
            "gpu_launches": int(st["kernel_launches"])}
    if rank == 0:
        print(json.dumps(line), flush=True)
    sk.close()
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.batch_only:
        print(json.dumps(run_batched(max(3, args.steps), args.warmup, args.batch_particles)))
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
