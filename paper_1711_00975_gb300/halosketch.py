"""ctypes binding of libhalosketch.so (include/halosketch.h), argument marshalling only.

Every function here forwards to the C entry point of the same name; arrays may
be torch tensors (device or host) or numpy arrays (host), passed by pointer.
All arithmetic of the path runs in the library's CUDA kernels; if the library
cannot be loaded the functions raise - there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_lock = threading.Lock()
_lib = None

HS_FLAG_SEARCH_SCAN = 1
HS_FLAG_SEARCH_DIRECTORY = 2
HS_FLAG_UPDATE_DIRECT = 4
HS_FLAG_UPDATE_BINNED = 8
HS_FLAG_DIR_INLINE = 16

HS_OK, HS_ERR_ARG, HS_ERR_CUDA, HS_ERR_OOM, HS_ERR_TABLE_FULL, HS_ERR_TIMEOUT, HS_ERR_STATE = range(7)
_NAMES = ["HS_OK", "HS_ERR_ARG", "HS_ERR_CUDA", "HS_ERR_OOM", "HS_ERR_TABLE_FULL",
          "HS_ERR_TIMEOUT", "HS_ERR_STATE"]


class HSError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        super().__init__(f"{where}: {_NAMES[status] if 0 <= status < 7 else status}: {msg}")


class hs_params(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_uint32), ("log2_width", ctypes.c_uint32),
                ("box", ctypes.c_double), ("cell", ctypes.c_double),
                ("hash_seed", ctypes.c_uint64), ("sample_seed", ctypes.c_uint64),
                ("flags", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class hs_info(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_uint32), ("log2_width", ctypes.c_uint32),
                ("grid", ctypes.c_uint32), ("inv_cell", ctypes.c_float),
                ("width", ctypes.c_uint64), ("n_cells", ctypes.c_uint64),
                ("n_seen", ctypes.c_uint64)]


class hs_tune(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_uint32), ("slot", ctypes.c_uint32),
                ("configs_tried", ctypes.c_uint32), ("best_ms", ctypes.c_float),
                ("window_volumes", ctypes.c_uint32)]


class hs_stats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_uint64), ("update_launches", ctypes.c_uint64),
                ("update_ms", ctypes.c_double), ("search_launches", ctypes.c_uint64),
                ("search_ms", ctypes.c_double), ("topk_ms", ctypes.c_double),
                ("topk_calls", ctypes.c_uint64), ("last_candidates", ctypes.c_uint64),
                ("last_threshold", ctypes.c_int32), ("last_passes", ctypes.c_uint32),
                ("flush_launches", ctypes.c_uint64), ("flush_ms", ctypes.c_double),
                ("h2d_bytes", ctypes.c_uint64), ("h2d_ms", ctypes.c_double),
                ("host_path_volumes", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


def library_path() -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "libhalosketch.so")


def lib():
    """Load libhalosketch.so (building it first when stale and nvcc is present)."""
    global _lib
    with _lock:
        if _lib is None:
            from . import build as _build
            path = library_path()
            try:
                path = _build.build()
            except (OSError, RuntimeError) as e:   # no nvcc: use a library built earlier
                if not os.path.exists(path):
                    raise RuntimeError(f"libhalosketch.so is not built and cannot be: {e}")
            L = ctypes.CDLL(path)
            vp, u32, u64, i32, f64, ci = (ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64,
                                          ctypes.c_int32, ctypes.c_double, ctypes.c_int)
            sig = {
                "sketch_create": [ctypes.POINTER(hs_params), vp, ctypes.POINTER(vp)],
                "sketch_update": [vp, vp, u64, f64],
                "sketch_set_hierarchy": [vp, u32, u32, u32],
                "sketch_super": [vp, ctypes.POINTER(vp)],
                "sketch_wait_copies": [vp],
                "sketch_update_packed": [vp, vp, u64, f64],
                "pack_positions": [vp, u64, f64, vp, vp],
                "sketch_query": [vp, vp, u64, vp],
                "topk_extract": [vp, u32, vp, vp, ctypes.POINTER(u32)],
                "sketch_destroy": [vp],
                "sketch_reset": [vp],
                "sketch_counters": [vp, vp],
                "sketch_load_counters": [vp, vp],
                "sketch_merge": [vp, vp],
                "sketch_info": [vp, ctypes.POINTER(hs_info)],
                "sketch_synchronize": [vp],
                "sketch_flush": [vp],
                "sketch_seek": [vp, u64],
                "sketch_stats": [vp, ctypes.POINTER(hs_stats), ci],
                "hs_measure_red_rate": [u64, u64, ctypes.POINTER(f64)],
                "sketch_query_noalloc": [vp, vp, u64, vp],
                "batch_create": [ctypes.POINTER(hs_params), u32, vp, vp, ctypes.POINTER(vp)],
                "batch_update": [vp, vp, vp, f64],
                "batch_topk": [vp, u32, vp, vp, vp],
                "batch_counters": [vp, u32, vp],
                "batch_reset": [vp],
                "batch_volume_info": [vp, u32, ctypes.POINTER(hs_info)],
                "batch_stats": [vp, ctypes.POINTER(hs_stats), ci],
                "batch_autotune": [vp, vp, vp, f64, ctypes.POINTER(hs_tune)],
                "batch_destroy": [vp],
                "mlp_create": [u64, vp, ctypes.POINTER(vp)],
                "mlp_set_params": [vp, vp],
                "mlp_get_params": [vp, vp],
                "mlp_forward": [vp, vp, u64, vp],
                "mlp_gradient": [vp, vp, vp, vp, u64, vp, vp],
                "mlp_train_step": [vp, vp, vp, vp, u64, ctypes.c_float, vp],
                "mlp_destroy": [vp],
                "exact_counts": [vp, u64, f64, f64, u32, vp, vp, vp, u64, ctypes.POINTER(u64)],
                "learned_create": [ctypes.POINTER(hs_params), u32, u32, u64, f64, vp,
                                   ctypes.POINTER(vp)],
                "exact_create": [f64, f64, u32, vp, ctypes.POINTER(vp)],
                "exact_add": [vp, vp, u64],
                "exact_list": [vp, vp, vp, u64, ctypes.POINTER(u64)],
                "exact_topk": [vp, u32, vp, vp, ctypes.POINTER(u32)],
                "exact_query": [vp, vp, u64, vp],
                "exact_reset": [vp],
                "exact_destroy": [vp],
                "learned_capacity": [vp, ctypes.POINTER(u64), ctypes.POINTER(u64)],
                "learned_routed": [vp, vp, u64, ctypes.POINTER(u64)],
                "learned_prepare": [vp, vp, u64, vp, ctypes.POINTER(u64)],
                "learned_sample": [vp, vp, u64],
                "learned_route": [vp, vp, ctypes.POINTER(u64)],
                "learned_update": [vp, vp, u64, f64],
                "learned_topk": [vp, u32, vp, vp, ctypes.POINTER(u32)],
                "learned_table": [vp, vp, vp, u64, ctypes.POINTER(u64)],
                "learned_logits": [vp, vp, vp, u64, ctypes.POINTER(u64)],
                "learned_features": [vp, vp, u64, ctypes.POINTER(u64)],
                "learned_coarse_counts": [vp, vp],
                "learned_sketch": [vp, ctypes.POINTER(vp)],
                "learned_reset": [vp],
                "learned_destroy": [vp],
            }
            for name, args in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            L.hs_last_error.argtypes = []
            L.hs_last_error.restype = ctypes.c_char_p
            _lib = L
    return _lib


def hs_last_error() -> str:
    return lib().hs_last_error().decode()


def _check(st: int, where: str):
    if st != HS_OK:
        raise HSError(st, where, hs_last_error())


def _ptr(a) -> int:
    """Address of a torch tensor or numpy array (None -> 0)."""
    if a is None:
        return 0
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _stream_ptr(stream) -> int:
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_params(rows: int, log2_width: int, box: float, cell: float, hash_seed: int = 0,
                sample_seed: int = 0, flags: int = 0) -> hs_params:
    return hs_params(rows, log2_width, box, cell, hash_seed, sample_seed, flags, 0)


# ---- the C entry points ----

def sketch_create(params: hs_params, stream=None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().sketch_create(ctypes.byref(params), _stream_ptr(stream), ctypes.byref(h)),
           "sketch_create")
    return h


def sketch_update(h, xyz, n: int | None = None, sample_rate: float = 1.0) -> None:
    if n is None:
        n = (xyz.numel() if hasattr(xyz, "numel") else xyz.size) // 3
    _check(lib().sketch_update(h, _ptr(xyz), n, sample_rate), "sketch_update")


def sketch_query(h, keys, est) -> None:
    m = keys.numel() if hasattr(keys, "numel") else keys.size
    _check(lib().sketch_query(h, _ptr(keys), m, _ptr(est)), "sketch_query")


HS_NOALLOC_QUERY_MAX = 262144


def sketch_query_noalloc(h, keys, est) -> None:
    """sketch_query without device allocation (static library scratch, at most
    HS_NOALLOC_QUERY_MAX keys per call; see include/halosketch.h)."""
    m = keys.numel() if hasattr(keys, "numel") else keys.size
    _check(lib().sketch_query_noalloc(h, _ptr(keys), m, _ptr(est)), "sketch_query_noalloc")


def topk_extract(h, k: int, keys: np.ndarray, est: np.ndarray) -> int:
    n = ctypes.c_uint32()
    assert keys.size >= k and est.size >= k
    _check(lib().topk_extract(h, k, _ptr(keys), _ptr(est), ctypes.byref(n)), "topk_extract")
    return n.value


def sketch_destroy(h) -> None:
    _check(lib().sketch_destroy(h), "sketch_destroy")


def sketch_reset(h) -> None:
    _check(lib().sketch_reset(h), "sketch_reset")


def sketch_counters(h, out) -> None:
    _check(lib().sketch_counters(h, _ptr(out)), "sketch_counters")


def sketch_load_counters(h, src) -> None:
    _check(lib().sketch_load_counters(h, _ptr(src)), "sketch_load_counters")


def sketch_merge(dst, src) -> None:
    _check(lib().sketch_merge(dst, src), "sketch_merge")


def sketch_info(h) -> hs_info:
    info = hs_info()
    _check(lib().sketch_info(h, ctypes.byref(info)), "sketch_info")
    return info


def sketch_seek(h, n_seen: int) -> None:
    _check(lib().sketch_seek(h, n_seen), "sketch_seek")


def sketch_update_packed(h, records, n: int | None = None, sample_rate: float = 1.0) -> None:
    if n is None:
        n = records.numel() if hasattr(records, "numel") else records.size
    _check(lib().sketch_update_packed(h, _ptr(records), n, sample_rate), "sketch_update_packed")


def pack_positions(xyz, box: float, out, n: int | None = None, stream=None) -> None:
    """64-bit records of n float32 positions (device tensors)."""
    if n is None:
        n = xyz.numel() // 3
    _check(lib().pack_positions(_ptr(xyz), n, box, _stream_ptr(stream), _ptr(out)),
           "pack_positions")


def sketch_wait_copies(h) -> None:
    _check(lib().sketch_wait_copies(h), "sketch_wait_copies")


def sketch_flush(h) -> None:
    _check(lib().sketch_flush(h), "sketch_flush")


def sketch_synchronize(h) -> None:
    _check(lib().sketch_synchronize(h), "sketch_synchronize")


def sketch_stats(h, reset: bool = False) -> dict:
    s = hs_stats()
    _check(lib().sketch_stats(h, ctypes.byref(s), 1 if reset else 0), "sketch_stats")
    return s.as_dict()


def hs_measure_red_rate(n_counters: int, total_ops: int) -> float:
    r = ctypes.c_double()
    _check(lib().hs_measure_red_rate(n_counters, total_ops, ctypes.byref(r)), "hs_measure_red_rate")
    return r.value


# ---- convenience wrapper ----

class Sketch:
    """Owns one library handle; methods forward to the entry points above."""

    def __init__(self, rows: int, log2_width: int, box: float, cell: float, hash_seed: int = 0,
                 sample_seed: int = 0, stream=None, flags: int = 0):
        self.params = make_params(rows, log2_width, box, cell, hash_seed, sample_seed, flags)
        self.h = sketch_create(self.params, stream)
        info = sketch_info(self.h)
        self.rows, self.width, self.G, self.n_cells = info.rows, info.width, info.grid, info.n_cells

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            sketch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def update(self, xyz, n=None, rate: float = 1.0):
        sketch_update(self.h, xyz, n, rate)

    def update_packed(self, records, n=None, rate: float = 1.0):
        sketch_update_packed(self.h, records, n, rate)

    def query(self, keys) -> np.ndarray:
        keys = np.ascontiguousarray(keys, np.uint64)
        est = np.empty(keys.size, np.int32)
        sketch_query(self.h, keys, est)
        return est

    def topk(self, k: int):
        keys = np.empty(k, np.uint64)
        est = np.empty(k, np.int32)
        n = topk_extract(self.h, k, keys, est)
        return keys[:n], est[:n]

    def counters(self) -> np.ndarray:
        out = np.empty((self.rows, self.width), np.int32)
        sketch_counters(self.h, out)
        return out

    def load_counters(self, c: np.ndarray):
        c = np.ascontiguousarray(c, np.int32)
        assert c.shape == (self.rows, self.width)
        sketch_load_counters(self.h, c)

    def reset(self):
        sketch_reset(self.h)

    def merge(self, other: "Sketch"):
        sketch_merge(self.h, other.h)

    def info(self) -> hs_info:
        return sketch_info(self.h)

    def stats(self, reset=False) -> dict:
        return sketch_stats(self.h, reset)

    def synchronize(self):
        sketch_synchronize(self.h)

    def flush(self):
        sketch_flush(self.h)

    def set_hierarchy(self, super_factor: int, super_log2_width: int, c_mult: int = 2):
        """Count super-items of super_factor^3 cells too and query hierarchically."""
        _check(lib().sketch_set_hierarchy(self.h, super_factor, super_log2_width, c_mult),
               "sketch_set_hierarchy")

    def super_handle(self):
        out = ctypes.c_void_p()
        _check(lib().sketch_super(self.h, ctypes.byref(out)), "sketch_super")
        return out if out.value else None

    def super_counters(self) -> np.ndarray:
        sh = self.super_handle()
        info = sketch_info(sh)
        out = np.empty((info.rows, info.width), np.int32)
        sketch_counters(sh, out)
        return out

    def seek(self, n_seen: int):
        sketch_seek(self.h, n_seen)


# ---- batches of sub-volumes ----

def batch_create(params: hs_params, boxes, stream=None) -> ctypes.c_void_p:
    boxes = np.ascontiguousarray(boxes, np.float64)
    h = ctypes.c_void_p()
    _check(lib().batch_create(ctypes.byref(params), boxes.size, boxes.ctypes.data,
                              _stream_ptr(stream), ctypes.byref(h)), "batch_create")
    return h


def batch_update(b, xyz, offsets, sample_rate: float = 1.0) -> None:
    offsets = np.ascontiguousarray(offsets, np.uint64)
    _check(lib().batch_update(b, _ptr(xyz), offsets.ctypes.data, sample_rate), "batch_update")


def batch_topk(b, n_volumes: int, k: int):
    keys = np.empty(n_volumes * k, np.uint64)
    est = np.empty(n_volumes * k, np.int32)
    n = np.empty(n_volumes, np.uint32)
    _check(lib().batch_topk(b, k, keys.ctypes.data, est.ctypes.data, n.ctypes.data), "batch_topk")
    return [(keys[v * k:v * k + n[v]], est[v * k:v * k + n[v]]) for v in range(n_volumes)]


def batch_counters(b, volume: int, out) -> None:
    _check(lib().batch_counters(b, volume, _ptr(out)), "batch_counters")


def batch_reset(b) -> None:
    _check(lib().batch_reset(b), "batch_reset")


def batch_volume_info(b, volume: int) -> hs_info:
    info = hs_info()
    _check(lib().batch_volume_info(b, volume, ctypes.byref(info)), "batch_volume_info")
    return info


def batch_stats(b, reset: bool = False) -> dict:
    s = hs_stats()
    _check(lib().batch_stats(b, ctypes.byref(s), 1 if reset else 0), "batch_stats")
    return s.as_dict()


def batch_autotune(b, xyz, offsets, sample_rate: float = 1.0) -> dict:
    offsets = np.ascontiguousarray(offsets, np.uint64)
    t = hs_tune()
    _check(lib().batch_autotune(b, _ptr(xyz), offsets.ctypes.data, sample_rate, ctypes.byref(t)),
           "batch_autotune")
    return {f: getattr(t, f) for f, _ in t._fields_}


def batch_destroy(b) -> None:
    _check(lib().batch_destroy(b), "batch_destroy")


class Batch:
    """Owns one batch handle (independent sketches of several sub-volumes)."""

    def __init__(self, rows: int, log2_width: int, boxes, cell: float, hash_seed: int = 0,
                 sample_seed: int = 0, stream=None, flags: int = 0):
        self.boxes = np.ascontiguousarray(boxes, np.float64)
        box0 = float(self.boxes[0]) if self.boxes.size else 1.0
        self.params = make_params(rows, log2_width, box0, cell, hash_seed, sample_seed, flags)
        self.h = batch_create(self.params, self.boxes, stream)
        self.n = self.boxes.size
        self.rows, self.width = rows, 1 << log2_width

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def update(self, xyz, offsets, rate: float = 1.0):
        batch_update(self.h, xyz, offsets, rate)

    def topk(self, k: int):
        return batch_topk(self.h, self.n, k)

    def counters(self, volume: int) -> np.ndarray:
        out = np.empty((self.rows, self.width), np.int32)
        batch_counters(self.h, volume, out)
        return out

    def reset(self):
        batch_reset(self.h)

    def info(self, volume: int) -> hs_info:
        return batch_volume_info(self.h, volume)

    def stats(self, reset=False) -> dict:
        return batch_stats(self.h, reset)

    def autotune(self, xyz, offsets, rate: float = 1.0) -> dict:
        return batch_autotune(self.h, xyz, offsets, rate)


# ---- learned router ----

HS_MLP_PARAMS = 6017
MLP_IN, MLP_H = 27, 64


class MLP:
    """The router network (27 -> 64 -> 64 -> 1); all math in library kernels."""

    def __init__(self, seed: int = 0, stream=None):
        h = ctypes.c_void_p()
        _check(lib().mlp_create(seed, _stream_ptr(stream), ctypes.byref(h)), "mlp_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        out = np.empty(HS_MLP_PARAMS, np.float32)
        _check(lib().mlp_get_params(self.h, out.ctypes.data), "mlp_get_params")
        return out

    def set_params(self, p) -> None:
        p = np.ascontiguousarray(p, np.float32)
        assert p.size == HS_MLP_PARAMS
        _check(lib().mlp_set_params(self.h, p.ctypes.data), "mlp_set_params")

    def forward(self, feats) -> np.ndarray:
        feats = feats if not isinstance(feats, np.ndarray) else np.ascontiguousarray(feats, np.uint16)
        n = (feats.numel() if hasattr(feats, "numel") else feats.size) // MLP_IN
        out = np.empty(n, np.float32)
        _check(lib().mlp_forward(self.h, _ptr(feats), n, out.ctypes.data), "mlp_forward")
        return out

    def gradient(self, feats, y, w):
        n = (feats.numel() if hasattr(feats, "numel") else feats.size) // MLP_IN
        grad = np.empty(HS_MLP_PARAMS, np.float32)
        loss = np.empty(1, np.float32)
        _check(lib().mlp_gradient(self.h, _ptr(feats), _ptr(y), _ptr(w), n, grad.ctypes.data,
                                  loss.ctypes.data), "mlp_gradient")
        return grad, float(loss[0])

    def train_step(self, feats, y, w, lr: float, want_loss: bool = True):
        n = (feats.numel() if hasattr(feats, "numel") else feats.size) // MLP_IN
        loss = ctypes.c_float()
        _check(lib().mlp_train_step(self.h, _ptr(feats), _ptr(y), _ptr(w), n, lr,
                                    ctypes.byref(loss) if want_loss else None), "mlp_train_step")
        return loss.value if want_loss else None


def exact_counts(xyz, n: int, box: float, cell: float, log2_slots: int, stream=None):
    """(keys, counts) of every occupied cell, computed on the GPU (device xyz)."""
    nn = ctypes.c_uint64()
    _check(lib().exact_counts(_ptr(xyz), n, box, cell, log2_slots, _stream_ptr(stream), None, None,
                              0, ctypes.byref(nn)), "exact_counts")
    cap = nn.value
    keys = np.empty(max(cap, 1), np.uint64)
    cnt = np.empty(max(cap, 1), np.int32)
    _check(lib().exact_counts(_ptr(xyz), n, box, cell, log2_slots, _stream_ptr(stream),
                              keys.ctypes.data, cnt.ctypes.data, cap, ctypes.byref(nn)),
           "exact_counts")
    return keys[:nn.value], cnt[:nn.value]


class Exact:
    """Exact per-cell counts in a device hash table (the exact algorithm)."""

    def __init__(self, box: float, cell: float, log2_slots: int, stream=None):
        h = ctypes.c_void_p()
        _check(lib().exact_create(box, cell, log2_slots, _stream_ptr(stream), ctypes.byref(h)),
               "exact_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().exact_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add(self, xyz, n: int | None = None):
        if n is None:
            n = (xyz.numel() if hasattr(xyz, "numel") else xyz.size) // 3
        _check(lib().exact_add(self.h, _ptr(xyz), n), "exact_add")

    def size(self) -> int:
        nn = ctypes.c_uint64()
        _check(lib().exact_list(self.h, None, None, 0, ctypes.byref(nn)), "exact_list")
        return nn.value

    def list(self):
        n = self.size()
        keys = np.empty(max(n, 1), np.uint64)
        cnt = np.empty(max(n, 1), np.int32)
        nn = ctypes.c_uint64()
        _check(lib().exact_list(self.h, keys.ctypes.data, cnt.ctypes.data, n, ctypes.byref(nn)),
               "exact_list")
        return keys[:nn.value], cnt[:nn.value]

    def topk(self, k: int):
        keys = np.empty(max(k, 1), np.uint64)
        cnt = np.empty(max(k, 1), np.int32)
        n = ctypes.c_uint32()
        _check(lib().exact_topk(self.h, k, keys.ctypes.data, cnt.ctypes.data, ctypes.byref(n)),
               "exact_topk")
        return keys[:n.value], cnt[:n.value]

    def query(self, keys) -> np.ndarray:
        keys = np.ascontiguousarray(keys, np.uint64)
        out = np.empty(max(keys.size, 1), np.int32)
        _check(lib().exact_query(self.h, keys.ctypes.data, keys.size, out.ctypes.data),
               "exact_query")
        return out[:keys.size]

    def reset(self):
        _check(lib().exact_reset(self.h), "exact_reset")

    def recall(self, method_keys, k: int) -> float:
        """count{c in method_keys[:k] : f_c >= f_(k)} / k, f_(k) the k-th largest count."""
        top = self.topk(k)[1]
        if k <= 0:
            return 1.0
        fk = int(top[k - 1]) if top.size >= k else 0
        if fk <= 0:
            return 0.0
        f = self.query(np.asarray(method_keys, np.uint64)[:k])
        return float(np.count_nonzero(f >= fk)) / k


class Learned:
    """Learned sketch: routed coarse cells counted exactly, the rest sketched."""

    def __init__(self, rows: int, log2_width: int, box: float, cell: float, hash_seed: int = 0,
                 sample_seed: int = 0, coarse_factor: int = 10, table_log2: int = 20,
                 feature_seed: int = 64, feature_rate: float = 1.0 / 64, stream=None,
                 flags: int = 0):
        self.params = make_params(rows, log2_width, box, cell, hash_seed, sample_seed, flags)
        h = ctypes.c_void_p()
        _check(lib().learned_create(ctypes.byref(self.params), coarse_factor, table_log2,
                                    feature_seed, feature_rate, _stream_ptr(stream),
                                    ctypes.byref(h)), "learned_create")
        self.h = h
        sk = ctypes.c_void_p()
        _check(lib().learned_sketch(self.h, ctypes.byref(sk)), "learned_sketch")
        self.sketch_h = sk
        info = sketch_info(sk)
        self.rows, self.width, self.G = info.rows, info.width, info.grid
        self.R = coarse_factor
        self.Gc = self.G // coarse_factor
        mr, tb = ctypes.c_uint64(), ctypes.c_uint64()
        _check(lib().learned_capacity(self.h, ctypes.byref(mr), ctypes.byref(tb)),
               "learned_capacity")
        self.max_routed, self.table_bytes = mr.value, tb.value

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().learned_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def prepare(self, xyz, mlp: MLP, n: int | None = None) -> int:
        if n is None:
            n = (xyz.numel() if hasattr(xyz, "numel") else xyz.size) // 3
        nr = ctypes.c_uint64()
        _check(lib().learned_prepare(self.h, _ptr(xyz), n, mlp.h, ctypes.byref(nr)), "learned_prepare")
        return nr.value

    def sample(self, xyz, n: int | None = None):
        if n is None:
            n = (xyz.numel() if hasattr(xyz, "numel") else xyz.size) // 3
        _check(lib().learned_sample(self.h, _ptr(xyz), n), "learned_sample")

    def route(self, mlp: MLP) -> int:
        nr = ctypes.c_uint64()
        _check(lib().learned_route(self.h, mlp.h, ctypes.byref(nr)), "learned_route")
        return nr.value

    def set_hierarchy(self, super_factor: int, super_log2_width: int, c_mult: int = 2):
        """Hierarchical query of the inner sketch; call before prepare/route."""
        _check(lib().sketch_set_hierarchy(self.sketch_h, super_factor, super_log2_width, c_mult),
               "sketch_set_hierarchy")

    def super_counters(self) -> np.ndarray:
        out = ctypes.c_void_p()
        _check(lib().sketch_super(self.sketch_h, ctypes.byref(out)), "sketch_super")
        info = sketch_info(out)
        arr = np.empty((info.rows, info.width), np.int32)
        sketch_counters(out, arr)
        return arr

    def update(self, xyz, n: int | None = None, rate: float = 1.0):
        if n is None:
            n = (xyz.numel() if hasattr(xyz, "numel") else xyz.size) // 3
        _check(lib().learned_update(self.h, _ptr(xyz), n, rate), "learned_update")

    def topk(self, k: int):
        keys = np.empty(k, np.uint64)
        est = np.empty(k, np.int32)
        n = ctypes.c_uint32()
        _check(lib().learned_topk(self.h, k, keys.ctypes.data, est.ctypes.data, ctypes.byref(n)),
               "learned_topk")
        return keys[:n.value], est[:n.value]

    def table(self):
        nn = ctypes.c_uint64()
        _check(lib().learned_table(self.h, None, None, 0, ctypes.byref(nn)), "learned_table")
        keys = np.empty(max(nn.value, 1), np.uint64)
        cnt = np.empty(max(nn.value, 1), np.int32)
        _check(lib().learned_table(self.h, keys.ctypes.data, cnt.ctypes.data, nn.value,
                                   ctypes.byref(nn)), "learned_table")
        o = np.argsort(keys[:nn.value])
        return keys[:nn.value][o], cnt[:nn.value][o]

    def routed(self) -> np.ndarray:
        nn = ctypes.c_uint64()
        _check(lib().learned_routed(self.h, None, 0, ctypes.byref(nn)), "learned_routed")
        out = np.empty(max(nn.value, 1), np.uint64)
        _check(lib().learned_routed(self.h, out.ctypes.data, nn.value, ctypes.byref(nn)),
               "learned_routed")
        return out[:nn.value]

    def logits(self):
        nn = ctypes.c_uint64()
        _check(lib().learned_logits(self.h, None, None, 0, ctypes.byref(nn)), "learned_logits")
        keys = np.empty(max(nn.value, 1), np.uint64)
        lg = np.empty(max(nn.value, 1), np.float32)
        _check(lib().learned_logits(self.h, keys.ctypes.data, lg.ctypes.data, nn.value,
                                    ctypes.byref(nn)), "learned_logits")
        return keys[:nn.value], lg[:nn.value]

    def features(self):
        nn = ctypes.c_uint64()
        _check(lib().learned_features(self.h, None, 0, ctypes.byref(nn)), "learned_features")
        f = np.empty((max(nn.value, 1), MLP_IN), np.uint16)
        _check(lib().learned_features(self.h, f.ctypes.data, nn.value, ctypes.byref(nn)),
               "learned_features")
        return f[:nn.value]

    def coarse_counts(self) -> np.ndarray:
        out = np.empty(self.Gc ** 3, np.int32)
        _check(lib().learned_coarse_counts(self.h, out.ctypes.data), "learned_coarse_counts")
        return out

    def counters(self) -> np.ndarray:
        out = np.empty((self.rows, self.width), np.int32)
        sketch_counters(self.sketch_h, out)
        return out

    def reset(self):
        _check(lib().learned_reset(self.h), "learned_reset")
