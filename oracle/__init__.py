"""CPU oracle for the Count Sketch halo-finder path (TEST INFRASTRUCTURE ONLY).

Plain restatement of arXiv:1711.00975's method: mesh reduction (Sec. 2.1),
index-hash Bernoulli sampling (Sec. 3.1), Count Sketch Add / Estimate
(Sec. 2.2), Count Sketch with Full Search (Algorithm 1) and the exact
algorithm of Sec. 4.2.  The arithmetic lives in `hs_oracle.c` (built with
gcc -ffp-contract=off); this module loads it with ctypes and offers numpy
wrappers, plus `hashref`, a width-generic statement of the hash family used to
pin the 64-bit one.

Only tests, the smoke check and the benchmark's CPU-baseline / reference legs
may import this package.  It shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

INVALID_KEY = np.uint64(0xFFFFFFFFFFFFFFFF)


def build(force: bool = False) -> str:
    """Compile liboracle.so in place (gcc, -O2 -ffp-contract=off, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u32, u64, i32, f32, f64, vp, ci = (ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32,
                                               ctypes.c_float, ctypes.c_double, ctypes.c_void_p,
                                               ctypes.c_int)
            sig = {
                "or_splitmix64_next": ([vp], u64),
                "or_splitmix64_at": ([u64, u64], u64),
                "or_derive_seeds": ([u64, u32, vp], None),
                "or_grid_size": ([f64, f64], u32),
                "or_inv_cell": ([f64], f32),
                "or_cell": ([f32, f32, f32, f32, u32, vp], ci),
                "or_keys": ([vp, u64, f32, u32, vp], None),
                "or_sample_threshold": ([f64], u64),
                "or_keep": ([u64, u64, f64], ci),
                "or_hash_row": ([vp, vp, u32, vp, vp], None),
                "or_sketch_update": ([vp, u32, u32, vp, vp, u64, u64, f32, u32, u64, f64, ci], ci),
                "or_estimate": ([vp, u32, u32, vp, vp, u64, u32, vp], None),
                "or_row_estimates": ([vp, u32, u32, vp, u64, u32, vp], None),
                "or_topk_range": ([vp, u32, u32, vp, u32, u64, u64, u32, vp, vp, ci], u64),
                "or_topk_full": ([vp, u32, u32, vp, u32, u32, vp, vp, ci], u64),
                "or_exact_counts": ([vp, u64, u64, f32, u32, u64, f64, vp, vp, u64], u64),
                "or_coarse_hist": ([vp, u64, u64, f32, u32, u32, u64, f64, vp], None),
                "or_bf16": ([f32], ctypes.c_uint16),
                "or_feature_of": ([i32], ctypes.c_uint16),
                "or_features": ([vp, u32, vp, u64, vp], None),
                "or_mlp_forward_f32": ([vp, vp, u64, vp], None),
                "or_learned_update": ([vp, u32, u32, vp, vp, u64, u64, f32, u32, u64, f64, vp, u32,
                                       vp, vp, u64], u64),
                "or_topk_unrouted": ([vp, u32, u32, vp, u32, vp, u32, u32, vp, vp], u64),
                "or_sketch_update_super": ([vp, u32, u32, vp, vp, u64, u64, f32, u32, u32, u64,
                                            f64], None),
                "or_topk_hier": ([vp, u32, u32, vp, vp, u32, u32, vp, u32, u32, u32, u32, vp, vp,
                                  ci], u64),
                "or_pack": ([vp, u64, f64, vp], None),
                "or_cell_packed": ([u64, u32, vp], ci),
                "or_sketch_update_packed": ([vp, u32, u32, vp, vp, u64, u64, u32, u32, u64, f64, ci],
                                            ci),
                "or_mlp_forward_f32_mt": ([vp, vp, u64, vp, ci], None),
                "or_learned_update_mt": ([vp, u32, u32, vp, vp, u64, u64, f32, u32, u64, f64, vp,
                                          u32, vp, vp, u64, ci], u64),
                "or_topk_hier_unrouted": ([vp, u32, u32, vp, vp, u32, u32, vp, u32, u32, u32, u32,
                                           vp, u32, vp, vp, ci], u64),
            }
            for name, (args, res) in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


class Params:
    """Sketch parameters in the oracle's own terms (mirrors the C-ABI's)."""

    def __init__(self, rows: int, log2_width: int, box: float, cell: float, hash_seed: int,
                 sample_seed: int = 0):
        lib = _load()
        self.rows = int(rows)
        self.log2_width = int(log2_width)
        self.box = float(box)
        self.cell = float(cell)
        self.hash_seed = int(hash_seed)
        self.sample_seed = int(sample_seed)
        self.G = int(lib.or_grid_size(self.box, self.cell))
        self.inv_cell = float(lib.or_inv_cell(self.cell))
        self.seeds = derive_seeds(self.hash_seed, self.rows)

    @property
    def width(self) -> int:
        return 1 << self.log2_width

    @property
    def n_cells(self) -> int:
        return self.G ** 3


# ---- splitmix64 ----

def splitmix64_sequence(seed: int, count: int) -> list[int]:
    lib = _load()
    st = ctypes.c_uint64(seed)
    return [int(lib.or_splitmix64_next(ctypes.byref(st))) for _ in range(count)]


def splitmix64_at(seed: int, g: int) -> int:
    return int(_load().or_splitmix64_at(seed, g))


def derive_seeds(hash_seed: int, rows: int) -> np.ndarray:
    out = np.empty(4 * rows, np.uint64)
    _load().or_derive_seeds(hash_seed, rows, _ptr(out))
    return out


# ---- mesh reduction ----

def cell_of(x: float, y: float, z: float, p: Params):
    c = np.zeros(3, np.uint32)
    ok = _load().or_cell(x, y, z, p.inv_cell, p.G, _ptr(c))
    return (int(c[0]), int(c[1]), int(c[2])) if ok else None


def keys_of(xyz: np.ndarray, p: Params) -> np.ndarray:
    xyz = np.ascontiguousarray(xyz, np.float32)
    n = xyz.size // 3
    out = np.empty(n, np.uint64)
    _load().or_keys(_ptr(xyz), n, p.inv_cell, p.G, _ptr(out))
    return out


def key_decode(key: int, G: int):
    return key % G, (key // G) % G, key // (G * G)


# ---- sampling ----

def sample_threshold(rate: float) -> int:
    return int(_load().or_sample_threshold(rate))


def keep(g: int, sample_seed: int, rate: float) -> bool:
    return bool(_load().or_keep(g, sample_seed, rate))


def keep_mask(g0: int, n: int, sample_seed: int, rate: float) -> np.ndarray:
    lib = _load()
    return np.fromiter((lib.or_keep(g0 + i, sample_seed, rate) for i in range(n)), np.bool_, n)


# ---- hashes ----

def hash_row(p: Params, row: int, c3) -> tuple[int, int]:
    c = np.array(c3, np.uint32)
    b = ctypes.c_uint32()
    s = ctypes.c_int32()
    _load().or_hash_row(p.seeds[4 * row:].ctypes.data, _ptr(c), p.log2_width, ctypes.byref(b),
                        ctypes.byref(s))
    return int(b.value), int(s.value)


# ---- sketch ----

def new_counters(p: Params) -> np.ndarray:
    return np.zeros((p.rows, p.width), np.int32)


def sketch_update(C: np.ndarray, p: Params, xyz: np.ndarray, g0: int = 0, rate: float = 1.0,
                  nthreads: int = 1) -> np.ndarray:
    """Add the particles of `xyz` (global indices g0..) into C in place."""
    assert C.dtype == np.int32 and C.flags.c_contiguous and C.shape == (p.rows, p.width)
    xyz = np.ascontiguousarray(xyz, np.float32)
    n = xyz.size // 3
    rc = _load().or_sketch_update(_ptr(C), p.rows, p.log2_width, _ptr(p.seeds), _ptr(xyz), n, g0,
                                  p.inv_cell, p.G, p.sample_seed, rate, nthreads)
    if rc:
        raise MemoryError("oracle sketch_update out of memory")
    return C


def estimate(C: np.ndarray, p: Params, keys) -> np.ndarray:
    keys = np.ascontiguousarray(keys, np.uint64)
    out = np.empty(keys.size, np.int32)
    _load().or_estimate(_ptr(C), p.rows, p.log2_width, _ptr(p.seeds), _ptr(keys), keys.size,
                        p.G, _ptr(out))
    return out


def row_estimates(C: np.ndarray, p: Params, key: int) -> np.ndarray:
    out = np.empty(p.rows, np.int32)
    _load().or_row_estimates(_ptr(C), p.rows, p.log2_width, _ptr(p.seeds), key, p.G, _ptr(out))
    return out


def topk_full(C: np.ndarray, p: Params, k: int, nthreads: int = 1, key_lo: int = 0,
              key_hi: int | None = None):
    """CSFS top-k over the dictionary [key_lo, key_hi): (keys, estimates), ranked."""
    if key_hi is None:
        key_hi = p.n_cells
    k = int(k)
    keys = np.empty(max(k, 1), np.uint64)
    est = np.empty(max(k, 1), np.int32)
    n = _load().or_topk_range(_ptr(C), p.rows, p.log2_width, _ptr(p.seeds), p.G, key_lo, key_hi, k,
                              _ptr(keys), _ptr(est), nthreads)
    return keys[:n].copy(), est[:n].copy()


# ---- packed records (64 bits: three 21-bit coordinates, bit 63 = invalid) ----

PACK_INVALID = np.uint64(1 << 63)


def pack(xyz: np.ndarray, box: float) -> np.ndarray:
    xyz = np.ascontiguousarray(xyz, np.float32)
    out = np.empty(xyz.size // 3, np.uint64)
    _load().or_pack(_ptr(xyz), out.size, box, _ptr(out))
    return out


def cell_packed(p: int, G: int):
    c = np.zeros(3, np.uint32)
    ok = _load().or_cell_packed(int(p), G, _ptr(c))
    return (int(c[0]), int(c[1]), int(c[2])) if ok else None


def sketch_update_packed(C: np.ndarray, p: Params, packed: np.ndarray, g0: int = 0,
                         rate: float = 1.0, nthreads: int = 1, F: int = 1,
                         fine: Params | None = None) -> np.ndarray:
    """Add packed records; for a super-item sketch pass its params as p, the
    fine mesh's params as fine and the super factor F."""
    packed = np.ascontiguousarray(packed, np.uint64)
    G = (fine or p).G
    rc = _load().or_sketch_update_packed(_ptr(C), p.rows, p.log2_width, _ptr(p.seeds),
                                         _ptr(packed), packed.size, g0, G, F, p.sample_seed, rate,
                                         nthreads)
    if rc:
        raise MemoryError("oracle sketch_update_packed out of memory")
    return C


# ---- hierarchy (Algorithm 3, CSHi) ----

def super_params(p: Params, F: int, log2_width: int, rows: int | None = None) -> Params:
    """The super-item sketch M1: cells of F x F x F, hash seed hash_seed + 1."""
    q = Params(rows or p.rows, log2_width, p.box, p.cell * F, p.hash_seed + 1, p.sample_seed)
    assert q.G * F == p.G
    return q


def sketch_update_super(C1: np.ndarray, p: Params, q: Params, F: int, xyz: np.ndarray,
                        g0: int = 0, rate: float = 1.0) -> np.ndarray:
    """Add the super-item (cell / F per axis; cells on p's fine mesh) of every kept particle."""
    assert C1.dtype == np.int32 and C1.shape == (q.rows, q.width)
    xyz = np.ascontiguousarray(xyz, np.float32)
    _load().or_sketch_update_super(_ptr(C1), q.rows, q.log2_width, _ptr(q.seeds), _ptr(xyz),
                                   xyz.size // 3, g0, p.inv_cell, p.G, F, p.sample_seed, rate)
    return C1


def topk_hier(C2: np.ndarray, p: Params, C1: np.ndarray, q: Params, F: int, k: int,
              c_mult: int, nthreads: int = 1):
    keys = np.empty(max(k, 1), np.uint64)
    est = np.empty(max(k, 1), np.int32)
    n = _load().or_topk_hier(_ptr(C2), p.rows, p.log2_width, _ptr(p.seeds), _ptr(C1), q.rows,
                             q.log2_width, _ptr(q.seeds), p.G, F, k, c_mult, _ptr(keys), _ptr(est),
                             nthreads)
    return keys[:n].copy(), est[:n].copy()


def exact_counts(xyz: np.ndarray, p: Params, g0: int = 0, rate: float = 1.0):
    """Exact per-cell counts of the kept particles (Sec. 4.2): (keys sorted, counts)."""
    xyz = np.ascontiguousarray(xyz, np.float32)
    n = xyz.size // 3
    cap = n + 1
    keys = np.empty(cap, np.uint64)
    cnt = np.empty(cap, np.uint32)
    D = _load().or_exact_counts(_ptr(xyz), n, g0, p.inv_cell, p.G, p.sample_seed, rate,
                                _ptr(keys), _ptr(cnt), cap)
    return keys[:D].copy(), cnt[:D].copy()


def exact_topk(keys: np.ndarray, counts: np.ndarray, k: int):
    """k heaviest cells by (count desc, key asc) from exact counts."""
    order = np.lexsort((keys, -counts.astype(np.int64)))
    sel = order[:k]
    return keys[sel], counts[sel]


def recall_at_k(method_keys: np.ndarray, exact_keys: np.ndarray, exact_cnt: np.ndarray,
                k: int) -> float:
    """count{c in method top-k : f_c >= f_(k)} / k, f_(k) = k-th largest exact count."""
    if k <= 0:
        return 1.0
    srt = np.sort(exact_cnt.astype(np.int64))[::-1]
    fk = srt[k - 1] if srt.size >= k else 0
    lut = dict(zip(exact_keys.tolist(), exact_cnt.tolist()))
    hit = sum(1 for key in method_keys[:k].tolist() if lut.get(key, 0) >= fk and fk > 0)
    return hit / k
