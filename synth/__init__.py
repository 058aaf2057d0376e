"""Seeded synthetic halo-populated boxes (inputs only).

The paper evaluates on Millennium / Millennium-XXL snapshots (arXiv:1711.00975,
Sec. 4.1 and 4.6), which are not available here.  These boxes stand in for
them: a periodic cube holding Plummer halos with a power-law mass function plus
a uniform background, emitted in a seeded pseudo-random stream order.  The
generator is index-addressable, so any slice of the stream can be produced on
its own (out-of-core chunks).

This module holds no part of the sketch method's arithmetic; both the CPU
oracle and the CUDA library consume what it produces.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "halobox.c")
_LIB = os.path.join(_HERE, "libhalobox.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile libhalobox.so in place with gcc (OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-D_GNU_SOURCE", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Config(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("box", ctypes.c_double), ("n_halo", ctypes.c_uint64),
                ("halo_frac", ctypes.c_double), ("m_min", ctypes.c_double),
                ("m_max", ctypes.c_double), ("slope", ctypes.c_double),
                ("r_scale", ctypes.c_double), ("m_pivot", ctypes.c_double),
                ("trunc", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("permute", ctypes.c_int32), ("pad", ctypes.c_int32)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp = ctypes.c_void_p
            lib.hb_build.argtypes = [ctypes.POINTER(_Config), ctypes.POINTER(vp)]
            lib.hb_build.restype = ctypes.c_int
            lib.hb_free.argtypes = [vp]
            lib.hb_generate.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint64, vp, ctypes.c_int]
            lib.hb_generate.restype = ctypes.c_int
            lib.hb_stream_index.argtypes = [vp, ctypes.c_uint64]
            lib.hb_stream_index.restype = ctypes.c_uint64
            lib.hb_n_in_halos.argtypes = [vp]
            lib.hb_n_in_halos.restype = ctypes.c_uint64
            lib.hb_catalogue.argtypes = [vp, vp, vp, vp, vp]
            _lib = lib
    return _lib


@dataclass
class BoxSpec:
    """Recipe of one synthetic box (sizes in Mpc/h)."""
    n: int
    box: float
    n_halo: int
    seed: int = 0
    halo_frac: float = 0.7
    m_min: float = 20.0
    m_max: float = 20000.0
    slope: float = 1.9
    r_scale: float = 0.05
    m_pivot: float = 1000.0
    trunc: float = 20.0
    permute: bool = True


class HaloBox:
    """A generated box; `generate(i0, count)` returns float32 xyz rows."""

    def __init__(self, spec: BoxSpec):
        self.spec = spec
        lib = _load()
        c = _Config(spec.n, spec.box, spec.n_halo, spec.halo_frac, spec.m_min, spec.m_max,
                    spec.slope, spec.r_scale, spec.m_pivot, spec.trunc, spec.seed,
                    1 if spec.permute else 0, 0)
        h = ctypes.c_void_p()
        rc = lib.hb_build(ctypes.byref(c), ctypes.byref(h))
        if rc != 0:
            raise ValueError(f"hb_build failed ({rc}) for {spec}")
        self._h = h
        self._lib = lib

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.hb_free(h)
            self._h = None

    @property
    def n(self) -> int:
        return self.spec.n

    @property
    def n_in_halos(self) -> int:
        return int(self._lib.hb_n_in_halos(self._h))

    def generate(self, i0: int = 0, count: int | None = None, out: np.ndarray | None = None,
                 nthreads: int = 0) -> np.ndarray:
        """float32 array (count, 3) of stream positions [i0, i0+count)."""
        if count is None:
            count = self.spec.n - i0
        if out is None:
            out = np.empty((count, 3), dtype=np.float32)
        assert out.dtype == np.float32 and out.flags.c_contiguous and out.size >= 3 * count
        rc = self._lib.hb_generate(self._h, i0, count, out.ctypes.data, nthreads)
        if rc != 0:
            raise ValueError("range outside the box's stream")
        return out

    def generate_into_ptr(self, ptr: int, i0: int, count: int, nthreads: int = 0) -> None:
        """Write stream positions [i0, i0+count) to a host address (e.g. pinned memory)."""
        rc = self._lib.hb_generate(self._h, i0, count, ctypes.c_void_p(ptr), nthreads)
        if rc != 0:
            raise ValueError("range outside the box's stream")

    def stream_index(self, i: int) -> int:
        return int(self._lib.hb_stream_index(self._h, i))

    def catalogue(self):
        H = self.spec.n_halo
        centre = np.empty((max(H, 1), 3), np.float64)
        mass = np.empty(max(H, 1), np.float64)
        a = np.empty(max(H, 1), np.float64)
        count = np.empty(max(H, 1), np.uint64)
        self._lib.hb_catalogue(self._h, centre.ctypes.data, mass.ctypes.data, a.ctypes.data,
                               count.ctypes.data)
        return centre[:H], mass[:H], a[:H], count[:H]


# ---------------------------------------------------------------------------
# Workload recipes.  Cell size 0.1 Mpc/h throughout; the uniform background is
# 30 % of the particles; halo masses follow dN/dM ~ M^-1.9 on [20, 20000].
# ---------------------------------------------------------------------------

def small_box(seed: int = 0) -> BoxSpec:
    """2^20 particles, 100 Mpc/h, 1000 halos."""
    return BoxSpec(n=1 << 20, box=100.0, n_halo=1000, seed=seed)


def scale_box(seed: int = 1, n: int = 10**9) -> BoxSpec:
    """10^9 particles, 500 Mpc/h, 10^6 halos (the Millennium-sized mesh)."""
    return BoxSpec(n=n, box=500.0, n_halo=10**6, seed=seed)


def training_box(seed: int) -> BoxSpec:
    """100 Mpc/h at the density of the 500 Mpc/h box: 8e6 particles, 8000 halos."""
    return BoxSpec(n=8 * 10**6, box=100.0, n_halo=8000, seed=seed)


def stream_box(seed: int = 4) -> BoxSpec:
    """2e10 particles, 2000 Mpc/h, 6.4e7 halos (out-of-core stream)."""
    return BoxSpec(n=2 * 10**10, box=2000.0, n_halo=64 * 10**6, seed=seed)


def subvolume_specs(seed: int = 3, count: int = 64, target_total: float = 3e8) -> list[BoxSpec]:
    """Uneven sub-volumes: counts log-uniform in [2^16, 2^26], rescaled so the
    total is about `target_total`; box side 25*(N/2^16)^(1/3) Mpc/h and
    round(1000*N/2^20) halos each."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(16.0, 26.0, size=count)
    n = 2.0 ** u
    lo, hi = 2.0 ** 16, 2.0 ** 26
    for _ in range(50):
        s = target_total / n.sum()
        if abs(s - 1.0) < 1e-3:
            break
        n = np.clip(n * s, lo, hi)
    specs = []
    for i, ni in enumerate(n):
        ni = int(round(ni))
        L = 25.0 * (ni / 2.0 ** 16) ** (1.0 / 3.0)
        L = round(L / 0.1) * 0.1   # a whole number of 0.1 Mpc/h cells
        specs.append(BoxSpec(n=ni, box=L, n_halo=max(1, int(round(1000 * ni / 2 ** 20))),
                             seed=seed * 1000 + i))
    return specs
