"""Seeded synthetic drift-chamber events (input generator only).

The paper evaluates on simulated STCF MDC samples with nominal background
(Sec. 4); those samples are not available, so this module generates events of
the same kind: 48 axial layers, circular tracks from the origin in a 1 T field,
uniform noise occupancy. It holds none of the Hough method's arithmetic and is
the one module both the CUDA path and the CPU oracle take inputs from.

The work is done by ``hough_gen.c`` (counter-based RNG, pthreads over events),
compiled here with gcc on first use.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hough_gen.c")
_OUT = os.path.join(_HERE, "_build", "libhough_gen.so")
_lock = threading.Lock()
_lib = None

N_LAYERS = 48
N_CELLS = 10656


class _Cfg(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("tracks_mode", ctypes.c_int32),
        ("tracks_a", ctypes.c_int32),
        ("tracks_b", ctypes.c_int32),
        ("pt_mode", ctypes.c_int32),
        ("tracks_mean", ctypes.c_double),
        ("pt_a", ctypes.c_double),
        ("pt_b", ctypes.c_double),
        ("pt_frac", ctypes.c_double),
        ("pt_a2", ctypes.c_double),
        ("pt_b2", ctypes.c_double),
        ("noise_mode", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("noise_a", ctypes.c_double),
        ("noise_b", ctypes.c_double),
    ]


@dataclass(frozen=True)
class EventConfig:
    """One synthetic workload: event distribution plus the Hough parameters it is run with."""

    name: str
    n_events: int
    seed: int
    tracks_mode: int
    tracks_a: int
    tracks_b: int
    tracks_mean: float
    pt_mode: int
    pt_a: float
    pt_b: float
    noise_mode: int
    noise_a: float
    noise_b: float
    n_theta: int
    n_rho: int
    threshold: int
    pt_frac: float = 0.0
    pt_a2: float = 0.0
    pt_b2: float = 0.0
    keep_halfwidth: int = 1
    max_peaks: int = 1024

    def cstruct(self) -> _Cfg:
        return _Cfg(
            seed=self.seed, tracks_mode=self.tracks_mode, tracks_a=self.tracks_a, tracks_b=self.tracks_b,
            pt_mode=self.pt_mode, tracks_mean=self.tracks_mean, pt_a=self.pt_a, pt_b=self.pt_b,
            pt_frac=self.pt_frac, pt_a2=self.pt_a2, pt_b2=self.pt_b2, noise_mode=self.noise_mode,
            reserved=0, noise_a=self.noise_a, noise_b=self.noise_b)


# The five workloads: plain small, plain paper-scale, batched, served (same event
# distribution as batched), high-occupancy stress. Seeds are 0x5EED0000 + index.
# max_peaks is sized above the largest peak count seen in each workload, so no
# event overflows its peak list.
CONFIGS = {
    "plain_small": EventConfig("plain_small", 100, 0x5EED0000, 0, 2, 2, 0.0, 0, 200.0, 1000.0, 0, 0.05, 0.05,
                               64, 64, 12),
    "plain_paper": EventConfig("plain_paper", 1000, 0x5EED0001, 1, 2, 8, 0.0, 1, 50.0, 1500.0, 0, 0.10, 0.10,
                               256, 256, 16, max_peaks=2048),
    "batched": EventConfig("batched", 100000, 0x5EED0002, 2, 0, 16, 4.0, 1, 50.0, 1500.0, 1, 0.05, 0.30,
                           256, 256, 16, max_peaks=4096),
    "served": EventConfig("served", 100000, 0x5EED0003, 2, 0, 16, 4.0, 1, 50.0, 1500.0, 1, 0.05, 0.30,
                          256, 256, 16, max_peaks=4096),
    "stress": EventConfig("stress", 10000, 0x5EED0004, 0, 16, 16, 0.0, 2, 120.0, 1500.0, 0, 0.40, 0.40,
                          512, 512, 20, pt_frac=0.4, pt_a2=50.0, pt_b2=120.0, max_peaks=16384),
    # the plain_paper events (same seed) at the paper's own discretisation, 1000 x 1000 (Sec. 2);
    # T = 12 keeps ~93 % of the track hits of these events, close to the paper's R_s
    "paper_1000": EventConfig("paper_1000", 1000, 0x5EED0001, 1, 2, 8, 0.0, 1, 50.0, 1500.0, 0, 0.10, 0.10,
                              1000, 1000, 12, max_peaks=1024),
}


def _build() -> str:
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    tmp = _OUT + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _OUT)
    return _OUT


def build() -> None:
    _load()


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(_build())
            i64p = ctypes.POINTER(ctypes.c_int64)
            i32p = ctypes.POINTER(ctypes.c_int32)
            f64p = ctypes.POINTER(ctypes.c_double)
            lib.hg_count.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_int64, ctypes.c_int64, i64p, ctypes.c_int]
            lib.hg_fill.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_int64, ctypes.c_int64, i64p, i32p, i32p,
                                    ctypes.c_int]
            lib.hg_event_tracks.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_int64, f64p, i32p, f64p, ctypes.c_int]
            lib.hg_geometry.argtypes = [i32p, i32p, i32p]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(ctypes.POINTER(t)) if a is not None else None


@dataclass
class Events:
    """Hits of a batch: ``xy`` int32 [n_hits, 2] in um, ``off`` int64 [n_events + 1], ``truth`` int32 [n_hits]
    (track index within the event, -1 for noise)."""

    xy: np.ndarray
    off: np.ndarray
    truth: np.ndarray | None

    @property
    def n_events(self) -> int:
        return len(self.off) - 1

    @property
    def n_hits(self) -> int:
        return int(self.off[-1])


def _threads(threads):
    return threads if threads else max(1, os.cpu_count() or 1)


def generate(cfg: EventConfig | str, n_events: int | None = None, first_event: int = 0, threads: int | None = None,
             with_truth: bool = True) -> Events:
    """Events ``[first_event, first_event + n_events)`` of workload ``cfg`` (deterministic in the seed)."""
    if isinstance(cfg, str):
        cfg = CONFIGS[cfg]
    n = cfg.n_events if n_events is None else int(n_events)
    lib = _load()
    c = cfg.cstruct()
    counts = np.zeros(n, dtype=np.int64)
    if n:
        rc = lib.hg_count(ctypes.byref(c), first_event, n, _ptr(counts, ctypes.c_int64), _threads(threads))
        if rc != 0:
            raise RuntimeError("hg_count failed")
    off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    xy = np.empty((int(off[-1]), 2), dtype=np.int32)
    truth = np.empty(int(off[-1]), dtype=np.int32) if with_truth else None
    if n:
        rc = lib.hg_fill(ctypes.byref(c), first_event, n, _ptr(off, ctypes.c_int64), _ptr(xy, ctypes.c_int32),
                         _ptr(truth, ctypes.c_int32) if truth is not None else None, _threads(threads))
        if rc != 0:
            raise RuntimeError("hg_fill failed")
    return Events(xy=xy, off=off, truth=truth)


def event_tracks(cfg: EventConfig | str, event: int):
    """Truth tracks of one event: list of (pT MeV/c, charge, phi0 rad)."""
    if isinstance(cfg, str):
        cfg = CONFIGS[cfg]
    lib = _load()
    c = cfg.cstruct()
    pt = np.zeros(64)
    q = np.zeros(64, dtype=np.int32)
    phi0 = np.zeros(64)
    n = lib.hg_event_tracks(ctypes.byref(c), event, _ptr(pt, ctypes.c_double), _ptr(q, ctypes.c_int32),
                            _ptr(phi0, ctypes.c_double), 64)
    return [(float(pt[i]), int(q[i]), float(phi0[i])) for i in range(min(n, 64))]


def geometry():
    """Wire table: (wire_x int32 [10656], wire_y int32 [10656], layer_first int32 [49])."""
    lib = _load()
    wx = np.zeros(N_CELLS, dtype=np.int32)
    wy = np.zeros(N_CELLS, dtype=np.int32)
    lf = np.zeros(N_LAYERS + 1, dtype=np.int32)
    lib.hg_geometry(_ptr(wx, ctypes.c_int32), _ptr(wy, ctypes.c_int32), _ptr(lf, ctypes.c_int32))
    return wx, wy, lf


def concat(parts: list[Events]) -> Events:
    """Concatenates batches (offsets re-based)."""
    xs, offs, ts = [], [np.zeros(1, dtype=np.int64)], []
    base = 0
    for p in parts:
        xs.append(p.xy)
        offs.append(p.off[1:] + base)
        ts.append(p.truth if p.truth is not None else np.full(p.n_hits, -1, np.int32))
        base += p.n_hits
    return Events(xy=np.concatenate(xs) if xs else np.zeros((0, 2), np.int32), off=np.concatenate(offs),
                  truth=np.concatenate(ts) if ts else np.zeros(0, np.int32))
