"""CPU oracle of the conformal Hough hit filter -- TEST INFRASTRUCTURE ONLY.

Plain C loops (``hough_oracle.c``, compiled with gcc on first use) restating the
paper's method step by step: conformal map Eq. (1) (with the factor 2 that makes
Eq. (2) hold), the rho matrix R of Sec. 3, integer voting, 3x3 peak finding and
back-projection hit selection (Sec. 2), the metrics Eq. (8)-(9). Only the tests,
``__graft_entry__.smoke()`` and the benchmark's ``cpu_baseline`` / reference leg
may import this package. It shares no code with the CUDA library.

Parity: every function here is pinned by ``tests/test_oracle_pins.py`` (closed
forms from Eq. (1)-(2), vote invariants, brute force against an independent
big-integer restatement, hand-built peak cases). The physics metrics R_c / R_s
are computed on synthetic events only; the paper's Table 1 values need its
simulated samples, so they are parity unpinned against the paper.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hough_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libhough_oracle.so")
_lock = threading.Lock()
_lib = None

F_BAD_HIT = 1
F_BAD_OFFSETS = 2
F_PEAK_OVERFLOW = 4
F_EVENT_TOO_LARGE = 8

PEAK_DTYPE = np.dtype([("theta_bin", "<i2"), ("rho_bin", "<i2"), ("votes", "<i2"), ("flags", "<i2")])


class Params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in (
        "n_theta", "n_rho", "threshold", "keep_halfwidth", "max_peaks", "theta_tiles", "events_per_cta", "block",
        "peak_mode", "rel_num", "rel_den", "nms_radius")]


PEAK_LOCAL_MAX, PEAK_ITERATIVE = 0, 1


def params(n_theta, n_rho, threshold, keep_halfwidth=1, max_peaks=1024, peak_mode=PEAK_LOCAL_MAX, rel_num=0,
           rel_den=1, nms_radius=1) -> Params:
    """Parameters; peak_mode 1 selects the iterative finder (relative threshold rel_num/rel_den of
    the accumulator maximum, suppression half-width nms_radius)."""
    return Params(n_theta, n_rho, threshold, keep_halfwidth, max_peaks, 0, 0, 0, peak_mode, rel_num, rel_den,
                  nms_radius)


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
            P = ctypes.POINTER
            i16p, i32p, i64p, u8p, u64p = (P(ctypes.c_int16), P(ctypes.c_int32), P(ctypes.c_int64),
                                           P(ctypes.c_uint8), P(ctypes.c_uint64))
            lib.or_tables.argtypes = [ctypes.c_int32, i16p, i16p]
            lib.or_map_hit.argtypes = [ctypes.c_int32, ctypes.c_int32, i64p, i64p]
            lib.or_map_hit.restype = ctypes.c_int32
            lib.or_rho.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int16, ctypes.c_int16]
            lib.or_rho.restype = ctypes.c_int64
            lib.or_bin.argtypes = [ctypes.c_int64, ctypes.c_int32]
            lib.or_bin.restype = ctypes.c_int32
            lib.or_peaks.argtypes = [i16p, P(Params), ctypes.c_void_p]
            lib.or_peaks.restype = ctypes.c_int32
            lib.or_peaks_iterative.argtypes = [i16p, P(Params), ctypes.c_void_p]
            lib.or_peaks_iterative.restype = ctypes.c_int32
            lib.or_checksum.argtypes = [i16p, ctypes.c_int32, ctypes.c_int32]
            lib.or_circles.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
            lib.or_circles.restype = None
            lib.or_checksum.restype = ctypes.c_uint64
            lib.or_run.argtypes = [i32p, ctypes.c_int64, i64p, ctypes.c_int64, P(Params), i16p, i32p,
                                   ctypes.c_void_p, u8p, i32p, u64p, ctypes.c_int32]
            lib.or_run.restype = ctypes.c_int32
            lib.or_const_H.restype = ctypes.c_int64
            _lib = lib
    return _lib


def _p(a, t):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(t))


H = None


def const_H() -> int:
    return int(_load().or_const_H())


def tables(n_theta: int):
    c = np.zeros(n_theta, np.int16)
    s = np.zeros(n_theta, np.int16)
    _load().or_tables(n_theta, _p(c, ctypes.c_int16), _p(s, ctypes.c_int16))
    return c, s


def map_hit(x: int, y: int):
    """(status, u_q, v_q) of one hit."""
    u = ctypes.c_int64()
    v = ctypes.c_int64()
    st = _load().or_map_hit(int(x), int(y), ctypes.byref(u), ctypes.byref(v))
    return int(st), int(u.value), int(v.value)


def rho(uq: int, vq: int, c: int, s: int) -> int:
    return int(_load().or_rho(uq, vq, c, s))


def bin_of(rho_q: int, n_rho: int) -> int:
    return int(_load().or_bin(int(rho_q), int(n_rho)))


def peaks(acc: np.ndarray, p: Params):
    """Peaks of one accumulator [n_theta, n_rho] int16: (true count, stored peak records)."""
    acc = np.ascontiguousarray(acc, dtype=np.int16)
    out = np.zeros(max(p.max_peaks, 1), dtype=PEAK_DTYPE)
    n = _load().or_peaks(_p(acc, ctypes.c_int16), ctypes.byref(p), out.ctypes.data)
    return int(n), out[: min(n, p.max_peaks)]


def peaks_iterative(acc: np.ndarray, p: Params):
    """Iterative peaks of one accumulator [n_theta, n_rho] int16: (true count, stored records in
    extraction order)."""
    acc = np.ascontiguousarray(acc, dtype=np.int16)
    out = np.zeros(max(p.max_peaks, 1), dtype=PEAK_DTYPE)
    n = _load().or_peaks_iterative(_p(acc, ctypes.c_int16), ctypes.byref(p), out.ctypes.data)
    return int(n), out[: min(n, p.max_peaks)]


def checksum(acc: np.ndarray) -> int:
    acc = np.ascontiguousarray(acc, dtype=np.int16)
    return int(_load().or_checksum(_p(acc, ctypes.c_int16), acc.shape[0], acc.shape[1]))


def circles(peaks: np.ndarray, n_theta: int, n_rho: int, b_tesla: float = 1.0) -> np.ndarray:
    """Eq. (2) circle of each peak record (PEAK_DTYPE array): float64 [n, 4] = x_c mm, y_c mm,
    r_c mm, pT MeV/c, at the bin centres."""
    pk = np.ascontiguousarray(peaks, dtype=PEAK_DTYPE).reshape(-1)
    out = np.zeros((len(pk), 4), np.float64)
    if len(pk):
        _load().or_circles(pk.ctypes.data, len(pk), int(n_theta), int(n_rho), float(b_tesla),
                           _p(out, ctypes.c_double))
    return out


@dataclass
class Result:
    status: int
    npeaks: np.ndarray  # int32 [n_events], true counts
    peaks: np.ndarray  # PEAK_DTYPE [n_events, max_peaks], zero past the stored ones
    mask: np.ndarray  # uint8 [n_hits]
    nkept: np.ndarray  # int32 [n_events]
    checksum: np.ndarray  # uint64 [n_events]
    acc: np.ndarray | None  # int16 [n_events, n_theta, n_rho]


def run(xy: np.ndarray, off: np.ndarray, p: Params, with_acc: bool = False, threads: int = 1) -> Result:
    """Whole batch through the oracle (events split over ``threads`` host threads)."""
    lib = _load()
    xy = np.ascontiguousarray(xy, dtype=np.int32).reshape(-1, 2)
    off = np.ascontiguousarray(off, dtype=np.int64)
    ne = len(off) - 1
    nh = xy.shape[0]
    npk = np.zeros(ne, np.int32)
    pk = np.zeros((ne, p.max_peaks), PEAK_DTYPE)
    mask = np.zeros(nh, np.uint8)
    nkept = np.zeros(ne, np.int32)
    cs = np.zeros(ne, np.uint64)
    acc = np.zeros((ne, p.n_theta, p.n_rho), np.int16) if with_acc else None
    st = lib.or_run(_p(xy, ctypes.c_int32), nh, _p(off, ctypes.c_int64), ne, ctypes.byref(p),
                    _p(acc, ctypes.c_int16), _p(npk, ctypes.c_int32), pk.ctypes.data, _p(mask, ctypes.c_uint8),
                    _p(nkept, ctypes.c_int32), _p(cs, ctypes.c_uint64), int(threads))
    return Result(int(st), npk, pk, mask, nkept, cs, acc)


def metrics(mask: np.ndarray, truth: np.ndarray):
    """Eq. (8) R_c = N_select / N_total and Eq. (9) R_s = N_true,select / N_true."""
    n_total = len(mask)
    n_sel = int(mask.sum())
    true = truth >= 0
    n_true = int(true.sum())
    n_true_sel = int((mask.astype(bool) & true).sum())
    return (n_sel / n_total if n_total else 0.0), (n_true_sel / n_true if n_true else 0.0)
