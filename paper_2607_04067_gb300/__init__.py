"""GB300 conformal Hough hit filter: thin Python binding over ``libhough.so``.

Every step runs in the library's sm_103a kernels; this module only marshals
torch CUDA tensors (device memory, streams) into the C ABI of
``include/hough.h``. There is no CPU fallback: if the library cannot be built
or loaded, or a tensor is not on a CUDA device, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading
from dataclasses import dataclass

from . import _build

_lock = threading.Lock()
_lib = None

OK, EINVAL, EPARAM, ESMEM, ECUDA, EWORKSPACE, ETIMEDOUT, EFULL, EDEVICE = 0, -1, -2, -3, -4, -5, -6, -7, -8
F_BAD_HIT, F_BAD_OFFSETS, F_PEAK_OVERFLOW, F_EVENT_TOO_LARGE, F_TIMEOUT, F_LAUNCH_FAILED = 1, 2, 4, 8, 16, 32
STATUS_WORDS = 4
MAX_EVENT_HITS = 32767
HEADER = os.path.join(_build.ROOT, "include", "hough.h")


class HoughError(RuntimeError):
    def __init__(self, fn: str, code: int):
        lib = load()
        msg = lib.hough_strerror(code).decode()
        if code == ECUDA:
            msg += f" (cudaError {lib.hough_last_cuda_error()})"
        super().__init__(f"{fn}: {msg} [{code}]")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in (
        "n_theta", "n_rho", "threshold", "keep_halfwidth", "max_peaks", "theta_tiles", "events_per_cta", "block",
        "peak_mode", "rel_num", "rel_den", "nms_radius")]

    def __repr__(self):
        return "Params(" + ", ".join(f"{n}={getattr(self, n)}" for n, _ in self._fields_) + ")"


class ServeConfig(ctypes.Structure):
    _fields_ = [("params", Params), ("slots", ctypes.c_int32), ("max_batch_events", ctypes.c_int32),
                ("max_batch_hits", ctypes.c_int64), ("flush_ns", ctypes.c_int64), ("queue_capacity", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class ServeStall(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "count", "max_gap_ns", "max_gap_at", "user_ns", "sys_ns", "minor_faults", "voluntary_switches",
        "involuntary_switches")]


class ServeStats(ctypes.Structure):
    _fields_ = [("passes", ctypes.c_int64), ("batches", ctypes.c_int64), ("stall_ns", ctypes.c_int64),
                ("loop", ServeStall), ("submit", ServeStall)]


RESULT_DTYPE = [("id", "<i8"), ("status", "<i4"), ("npeaks", "<i4"), ("nkept", "<i4"), ("reserved", "<i4"),
                ("t_arrival_ns", "<i8"), ("t_done_ns", "<i8")]
BATCH_RECORD_DTYPE = [("t_gather", "<i8"), ("t_launched", "<i8"), ("t_done_seen", "<i8"), ("t_finished", "<i8"),
                      ("n_hits", "<i8"), ("n_events", "<i4"), ("slot", "<i4")]
SERVE_RECORDS = 65536


class ServeResult(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int32), ("npeaks", ctypes.c_int32),
                ("nkept", ctypes.c_int32), ("reserved", ctypes.c_int32), ("t_arrival_ns", ctypes.c_int64),
                ("t_done_ns", ctypes.c_int64)]


PEAK_LOCAL_MAX, PEAK_ITERATIVE = 0, 1
# HOUGH_PHASE_* of include/hough.h, in order
PHASES = ("clear", "stage", "vote", "fold", "scan", "exscan", "records", "merge", "it_max", "it_collect",
          "it_resolve", "it_order", "sel_columns", "sel_bitmaps", "sel_a", "sel_b")


def params(n_theta: int, n_rho: int, threshold: int, keep_halfwidth: int = 1, max_peaks: int = 1024,
           theta_tiles: int = 0, events_per_cta: int = 0, block: int = 0, peak_mode: int = PEAK_LOCAL_MAX,
           rel_num: int = 0, rel_den: int = 1, nms_radius: int = 1) -> Params:
    """Parameters of the path; peak_mode PEAK_ITERATIVE selects the paper's iterative finder
    (relative threshold rel_num/rel_den of the maximum, suppression half-width nms_radius)."""
    return Params(n_theta, n_rho, threshold, keep_halfwidth, max_peaks, theta_tiles, events_per_cta, block,
                  peak_mode, rel_num, rel_den, nms_radius)


def declared_symbols() -> list[str]:
    """Names of the entry points declared in include/hough.h."""
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w]+\s*\*?\s*(hough_\w+)\s*\(", text, flags=re.M)))


def load(build: bool = True):
    """Loads (building first if sources changed) libhough.so."""
    global _lib
    with _lock:
        if _lib is None:
            # HOUGH_PHASE_TIMERS=1 selects the phase-timer build (same results, per-phase cycles)
            variant = "phase" if os.environ.get("HOUGH_PHASE_TIMERS") == "1" else None
            path = _build.build(variant=variant) if build else _build.lib_path(variant)
            lib = ctypes.CDLL(path)
            vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
            P = ctypes.POINTER(Params)
            sig = {
                "hough_map": [vp, i64, vp, i64, vp, vp, vp, vp],
                "hough_vote": [vp, vp, i64, vp, i64, P, vp, vp, vp],
                "hough_peaks": [vp, i64, P, vp, vp, vp, vp],
                "hough_select": [vp, vp, i64, vp, i64, P, vp, vp, vp, vp, vp, vp],
                "hough_run": [vp, i64, vp, i64, P, vp, vp, vp, vp, vp, vp, ctypes.c_size_t, vp, vp],
                "hough_run_batched": [vp, i64, vp, i64, P, vp, vp, vp, vp, vp, vp, ctypes.c_size_t, vp, vp],
                "hough_resolve_params": [P],
                "hough_status": [vp, vp, ctypes.POINTER(i32)],
                "hough_last_cuda_error": [],
                "hough_selftest_bin": [i32, i64, i64, vp, vp],
                "hough_selftest_fpbin": [i32, i32, ctypes.c_uint64, i64, vp, vp],
                "hough_probe_smem_atomics": [i32, i32, i32, i32, i32, vp, vp],
                "hough_run_host": [vp, i64, vp, i64, P, vp, vp, vp, i64, vp, vp, vp, ctypes.c_size_t, vp, vp],
                "hough_run_batched_static": [vp, i64, vp, i64, P, vp, vp, vp, vp, vp, vp, vp],
                "hough_autotune": [P, vp, i64, vp, i64, vp, ctypes.c_size_t, vp, vp, ctypes.POINTER(ctypes.c_float)],
                "hough_circles": [vp, vp, i64, P, ctypes.c_double, vp, vp],
                "hough_phase_cycles": [vp, i32, i32, vp],
            }
            for name, args in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            lib.hough_workspace_size.argtypes = [P, i64]
            lib.hough_workspace_size.restype = ctypes.c_size_t
            SP = ctypes.POINTER(ServeConfig)
            for name, args in {
                "hough_serve_buffer_sizes": [SP, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)],
                "hough_serve_open": [SP, vp, ctypes.c_size_t, vp, ctypes.c_size_t, ctypes.POINTER(vp)],
                "hough_serve_submit": [vp, vp, i64, i64, vp, vp],
                "hough_serve_poll": [vp, vp, i32, ctypes.POINTER(i32)],
                "hough_serve_drain": [vp, i64],
                "hough_serve_replay": [vp, vp, vp, i64, vp, i64, ctypes.POINTER(i64), vp, vp, vp],
                "hough_serve_close": [vp],
                "hough_serve_trace": [vp, ctypes.POINTER(ServeStats), vp, i32, ctypes.POINTER(i32)],
                "hough_serve_inject_launch_failures": [vp, i32],
            }.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            lib.hough_autotune_scratch_size.argtypes = [P, i64, i64]
            lib.hough_autotune_scratch_size.restype = ctypes.c_size_t
            lib.hough_host_buffer_size.argtypes = [P, i64, i64]
            lib.hough_host_buffer_size.restype = ctypes.c_size_t
            lib.hough_set_stage_events.argtypes = [vp, vp]
            lib.hough_set_stage_events.restype = None
            lib.hough_set_host_timing.argtypes = [i32]
            lib.hough_set_host_timing.restype = None
            lib.hough_host_stage_ms.argtypes = [vp, i32]
            lib.hough_host_stage_ms.restype = ctypes.c_int
            lib.hough_strerror.argtypes = [ctypes.c_int]
            lib.hough_strerror.restype = ctypes.c_char_p
            _lib = lib
    return _lib


# ---------------------------------------------------------------- torch marshalling

def _torch():
    import torch
    return torch


def _dev(t, name, dtype=None):
    torch = _torch()
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    return t


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check(fn, rc):
    if rc != OK:
        raise HoughError(fn, rc)


def new_status(device="cuda"):
    torch = _torch()
    return torch.zeros(STATUS_WORDS, dtype=torch.int32, device=device)


def status(st, stream=None) -> int:
    """Synchronises the stream and returns the sticky device flags (word 0)."""
    flags = ctypes.c_int32(0)
    rc = load().hough_status(_ptr(_dev(st, "status", _torch().int32)), _stream(stream), ctypes.byref(flags))
    if rc not in (OK, EDEVICE):
        raise HoughError("hough_status", rc)
    return int(flags.value)


def resolve(p: Params) -> Params:
    q = Params(*[getattr(p, n) for n, _ in Params._fields_])
    _check("hough_resolve_params", load().hough_resolve_params(ctypes.byref(q)))
    return q


def workspace_size(p: Params, n_events: int) -> int:
    return int(load().hough_workspace_size(ctypes.byref(p), int(n_events)))


def workspace(p: Params, n_events: int, device="cuda"):
    torch = _torch()
    return torch.empty(workspace_size(p, n_events), dtype=torch.uint8, device=device)


# ---------------------------------------------------------------- stepwise calls

def map_hits(xy, off, st, uq=None, vq=None, stream=None):
    torch = _torch()
    xy = _dev(xy, "xy", torch.int32)
    off = _dev(off, "off", torch.int64)
    n = xy.shape[0]
    uq = torch.empty(n, dtype=torch.int64, device=xy.device) if uq is None else _dev(uq, "uq", torch.int64)
    vq = torch.empty(n, dtype=torch.int64, device=xy.device) if vq is None else _dev(vq, "vq", torch.int64)
    _check("hough_map", load().hough_map(_ptr(xy), n, _ptr(off), off.shape[0] - 1, _ptr(uq), _ptr(vq), _ptr(st),
                                         _stream(stream)))
    return uq, vq


def vote(uq, vq, off, p: Params, st, acc=None, stream=None):
    torch = _torch()
    ne = off.shape[0] - 1
    if acc is None:
        acc = torch.empty((ne, p.n_theta, p.n_rho), dtype=torch.int16, device=uq.device)
    _check("hough_vote", load().hough_vote(_ptr(_dev(uq, "uq", torch.int64)), _ptr(_dev(vq, "vq", torch.int64)),
                                           uq.shape[0], _ptr(_dev(off, "off", torch.int64)), ne, ctypes.byref(p),
                                           _ptr(_dev(acc, "acc", torch.int16)), _ptr(st), _stream(stream)))
    return acc


def peaks(acc, p: Params, st, npeaks=None, pk=None, stream=None):
    torch = _torch()
    ne = acc.shape[0]
    if npeaks is None:
        npeaks = torch.zeros(ne, dtype=torch.int32, device=acc.device)
    if pk is None:
        pk = torch.zeros((ne, p.max_peaks, 4), dtype=torch.int16, device=acc.device)
    _check("hough_peaks", load().hough_peaks(_ptr(_dev(acc, "acc", torch.int16)), ne, ctypes.byref(p),
                                             _ptr(_dev(npeaks, "npeaks", torch.int32)),
                                             _ptr(_dev(pk, "peaks", torch.int16)), _ptr(st), _stream(stream)))
    return npeaks, pk


def select(uq, vq, off, p: Params, npeaks, pk, st, mask=None, nkept=None, stream=None):
    torch = _torch()
    ne = off.shape[0] - 1
    if mask is None:
        mask = torch.empty(uq.shape[0], dtype=torch.uint8, device=uq.device)
    if nkept is None:
        nkept = torch.empty(ne, dtype=torch.int32, device=uq.device)
    _check("hough_select", load().hough_select(
        _ptr(_dev(uq, "uq", torch.int64)), _ptr(_dev(vq, "vq", torch.int64)), uq.shape[0],
        _ptr(_dev(off, "off", torch.int64)), ne, ctypes.byref(p), _ptr(_dev(npeaks, "npeaks", torch.int32)),
        _ptr(_dev(pk, "peaks", torch.int16)), _ptr(_dev(mask, "mask", torch.uint8)),
        _ptr(_dev(nkept, "nkept", torch.int32)), _ptr(st), _stream(stream)))
    return mask, nkept


def circles(npeaks, peaks, p: Params, b_tesla: float = 1.0, out=None, stream=None):
    """Eq. (2) circle of every stored peak: float32 [n_events, max_peaks, 4] = x_c mm, y_c mm,
    r_c mm, pT MeV/c (entries past each event's stored peaks are left as they were)."""
    torch = _torch()
    npeaks = _dev(npeaks, "npeaks", torch.int32)
    ne = npeaks.shape[0]
    if out is None:
        out = torch.zeros((ne, p.max_peaks, 4), dtype=torch.float32, device=npeaks.device)
    _check("hough_circles", load().hough_circles(_ptr(npeaks), _ptr(_dev(peaks, "peaks", torch.int16)), ne,
                                                 ctypes.byref(p), float(b_tesla),
                                                 _ptr(_dev(out, "circles", torch.float32)), _stream(stream)))
    return out


# ---------------------------------------------------------------- fused calls

@dataclass
class Outputs:
    npeaks: "object"  # int32 [n_events]
    peaks: "object"  # int16 [n_events, max_peaks, 4]: theta_bin, rho_bin, votes, flags
    mask: "object"  # uint8 [n_hits]
    nkept: "object"  # int32 [n_events]
    checksum: "object"  # int64 view of uint64 [n_events], or None
    ws: "object"
    status: "object"


def alloc_outputs(n_hits: int, n_events: int, p: Params, checksum: bool = False, device="cuda") -> Outputs:
    torch = _torch()
    return Outputs(
        npeaks=torch.zeros(n_events, dtype=torch.int32, device=device),
        peaks=torch.zeros((n_events, p.max_peaks, 4), dtype=torch.int16, device=device),
        mask=torch.zeros(n_hits, dtype=torch.uint8, device=device),
        nkept=torch.zeros(n_events, dtype=torch.int32, device=device),
        checksum=torch.zeros(n_events, dtype=torch.int64, device=device) if checksum else None,
        ws=workspace(p, n_events, device),
        status=new_status(device),
    )


def _check_outputs(out: "Outputs", n_hits: int, n_events: int, p: Params, need_ws: bool):
    """The C ABI sees plain pointers: check every output tensor's device, type and size here."""
    torch = _torch()
    need = [("npeaks", out.npeaks, torch.int32, n_events), ("peaks", out.peaks, torch.int16, n_events * p.max_peaks * 4),
            ("mask", out.mask, torch.uint8, n_hits), ("nkept", out.nkept, torch.int32, n_events),
            ("status", out.status, torch.int32, 4)]
    if out.checksum is not None:
        need.append(("checksum", out.checksum, torch.int64, n_events))
    if need_ws:
        need.append(("ws", out.ws, torch.uint8, workspace_size(p, n_events)))
    for name, t, dtype, n in need:
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype:
            raise TypeError(f"out.{name} must be a CUDA {dtype} tensor")
        if t.numel() < n:
            raise ValueError(f"out.{name} holds {t.numel()} elements, {n} needed")


def run(xy, off, p: Params, out: Outputs | None = None, checksum: bool = False, batched: bool = False,
        stream=None) -> Outputs:
    """Whole path (map, rho, vote, peaks, select) in the fused kernel; ``batched`` uses the
    persistent work-queue launch replayed as a CUDA graph."""
    torch = _torch()
    xy = _dev(xy, "xy", torch.int32)
    off = _dev(off, "off", torch.int64)
    ne = off.shape[0] - 1
    if out is None:
        out = alloc_outputs(xy.shape[0], ne, p, checksum, xy.device)
    _check_outputs(out, xy.shape[0], ne, p, need_ws=False)
    fn = load().hough_run_batched if batched else load().hough_run
    rc = fn(_ptr(xy), xy.shape[0], _ptr(off), ne, ctypes.byref(p), _ptr(out.npeaks), _ptr(out.peaks), _ptr(out.mask),
            _ptr(out.nkept), _ptr(out.checksum), _ptr(out.ws), out.ws.numel(), _ptr(out.status), _stream(stream))
    _check("hough_run_batched" if batched else "hough_run", rc)
    return out


def run_static(xy, off, p: Params, out: Outputs, stream=None) -> Outputs:
    """The batched path through ``hough_run_batched_static``: no workspace from the caller, the
    scratch comes from the library's built-in device array (``out.ws`` is not used)."""
    torch = _torch()
    xy = _dev(xy, "xy", torch.int32)
    off = _dev(off, "off", torch.int64)
    _check_outputs(out, xy.shape[0], off.shape[0] - 1, p, need_ws=False)
    rc = load().hough_run_batched_static(
        _ptr(xy), xy.shape[0], _ptr(off), off.shape[0] - 1, ctypes.byref(p), _ptr(out.npeaks), _ptr(out.peaks),
        _ptr(out.mask), _ptr(out.nkept), _ptr(out.checksum), _ptr(out.status), _stream(stream))
    _check("hough_run_batched_static", rc)
    return out


class HostRunner:
    """End-to-end calls through ``hough_run_host``: host (pinned) inputs in, host results out,
    every copy inside the call. Owns the device staging buffer and the pinned result buffers."""

    def __init__(self, n_hits: int, n_events: int, p: Params, peaks_cap: int | None = None, device="cuda"):
        torch = _torch()
        self.p = p
        self.n_hits, self.n_events = int(n_hits), int(n_events)
        nbytes = int(load().hough_host_buffer_size(ctypes.byref(p), self.n_hits, self.n_events))
        self.dbuf = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.status = new_status(device)
        cap = self.n_events * p.max_peaks if peaks_cap is None else int(peaks_cap)
        self.npeaks = torch.zeros(self.n_events, dtype=torch.int32).pin_memory()
        self.peak_off = torch.zeros(self.n_events + 1, dtype=torch.int64).pin_memory()
        self.peaks = torch.zeros((max(cap, 1), 4), dtype=torch.int16).pin_memory()
        self.mask = torch.zeros(max(self.n_hits, 1), dtype=torch.uint8).pin_memory()
        self.nkept = torch.zeros(self.n_events, dtype=torch.int32).pin_memory()
        self.cap = cap

    STAGES = ("h2d", "kernels", "pack", "d2h", "peaks_d2h", "span")

    def stage_ms(self):
        """Per-stage device milliseconds of this thread's last call made with timing on (see
        set_host_timing): stage busy times summed over the chunks, and the call's span."""
        buf = (ctypes.c_float * len(self.STAGES))()
        _check("hough_host_stage_ms", load().hough_host_stage_ms(buf, len(self.STAGES)))
        return {k: float(buf[i]) for i, k in enumerate(self.STAGES)}

    def d2h_bytes(self) -> int:
        """Bytes the last call copied back (results)."""
        return 4 * self.n_events * 2 + 8 * (self.n_events + 1) + self.n_hits + 8 * int(self.peak_off[-1]) + 4

    def __call__(self, xy_host, off_host, stream=None) -> int:
        """Runs on pinned int32 [n_hits, 2] / int64 [n_events + 1] host tensors; returns the status flags."""
        rc = load().hough_run_host(
            ctypes.c_void_p(xy_host.data_ptr()), self.n_hits, ctypes.c_void_p(off_host.data_ptr()), self.n_events,
            ctypes.byref(self.p), _ptr(self.npeaks), _ptr(self.peak_off), _ptr(self.peaks), self.cap,
            _ptr(self.mask), _ptr(self.nkept), _ptr(self.dbuf), self.dbuf.numel(), _ptr(self.status), _stream(stream))
        if rc == EDEVICE:
            return int(self.status[0].item())
        _check("hough_run_host", rc)
        return 0


class Server:
    """Continuous-batching serving loop (``hough_serve_*``). The device and pinned buffers are
    torch tensors owned by this object; the loop itself is a native thread in the library."""

    def __init__(self, p: Params, slots: int = 4, max_batch_events: int = 256, max_batch_hits: int = 1 << 20,
                 flush_us: float = 50.0, queue_capacity: int = 1 << 16, device="cuda"):
        torch = _torch()
        self.cfg = ServeConfig(p, slots, max_batch_events, max_batch_hits, int(flush_us * 1000), queue_capacity, 0)
        lib = load()
        db, hb = ctypes.c_size_t(), ctypes.c_size_t()
        _check("hough_serve_buffer_sizes", lib.hough_serve_buffer_sizes(ctypes.byref(self.cfg), ctypes.byref(db),
                                                                         ctypes.byref(hb)))
        self.dbuf = torch.empty(db.value + 256, dtype=torch.uint8, device=device)
        self.hbuf = torch.empty(hb.value + 256, dtype=torch.uint8).pin_memory()
        d0 = (-self.dbuf.data_ptr()) % 256
        h0 = (-self.hbuf.data_ptr()) % 256
        self.handle = ctypes.c_void_p()
        _check("hough_serve_open", lib.hough_serve_open(
            ctypes.byref(self.cfg), ctypes.c_void_p(self.dbuf.data_ptr() + d0), db.value,
            ctypes.c_void_p(self.hbuf.data_ptr() + h0), hb.value, ctypes.byref(self.handle)))

    def submit(self, xy_host, req_id: int, mask_out=None, peaks_out=None) -> int:
        """xy_host: contiguous int32 [n, 2] CPU tensor/array kept alive until completion."""
        ptr = xy_host.data_ptr() if hasattr(xy_host, "data_ptr") else xy_host.ctypes.data
        n = xy_host.shape[0]
        mo = None if mask_out is None else ctypes.c_void_p(
            mask_out.data_ptr() if hasattr(mask_out, "data_ptr") else mask_out.ctypes.data)
        po = None if peaks_out is None else ctypes.c_void_p(
            peaks_out.data_ptr() if hasattr(peaks_out, "data_ptr") else peaks_out.ctypes.data)
        return load().hough_serve_submit(self.handle, ctypes.c_void_p(ptr), n, req_id, mo, po)

    def poll(self, max_results: int = 1 << 16):
        buf = (ServeResult * max_results)()
        n = ctypes.c_int32()
        rc = load().hough_serve_poll(self.handle, buf, max_results, ctypes.byref(n))
        if rc:
            raise HoughError("hough_serve_poll", rc)
        return [buf[i] for i in range(n.value)]

    def poll_numpy(self, max_results: int = 1 << 22):
        import numpy as np
        out = np.zeros(max_results, np.dtype(RESULT_DTYPE))
        n = ctypes.c_int32()
        rc = load().hough_serve_poll(self.handle, ctypes.c_void_p(out.ctypes.data), max_results, ctypes.byref(n))
        if rc:
            raise HoughError("hough_serve_poll", rc)
        return out[: n.value]

    def drain(self, timeout_s: float = 30.0):
        _check("hough_serve_drain", load().hough_serve_drain(self.handle, int(timeout_s * 1e9)))

    def replay(self, xy_pool, off_pool, arrival_ns, mask_out=None, peaks_out=None, results_out=None) -> int:
        """Submits request i = pool event i mod n at its scheduled time; returns t0 (ns). With
        mask_out (uint8, the requests' hit counts summed) and peaks_out (int16 [requests,
        max_peaks, 4]) numpy arrays, each request's results are copied there; with results_out
        (result_array(n)) request i's result record goes to results_out[i] instead of poll()."""
        t0 = ctypes.c_int64()
        mo = None if mask_out is None else ctypes.c_void_p(mask_out.ctypes.data)
        po = None if peaks_out is None else ctypes.c_void_p(peaks_out.ctypes.data)
        ro = None if results_out is None else ctypes.c_void_p(results_out.ctypes.data)
        _check("hough_serve_replay", load().hough_serve_replay(
            self.handle, ctypes.c_void_p(xy_pool.ctypes.data), ctypes.c_void_p(off_pool.ctypes.data),
            len(off_pool) - 1, ctypes.c_void_p(arrival_ns.ctypes.data), len(arrival_ns), ctypes.byref(t0), mo, po,
            ro))
        return t0.value

    @staticmethod
    def result_array(n: int):
        """A numpy array of n result records, written once (its pages faulted in now)."""
        import numpy as np
        out = np.empty(n, np.dtype(RESULT_DTYPE))
        out.view(np.uint8).fill(0)
        return out

    def trace(self, max_records: int = 65536):
        """(stats dict, numpy records of the most recent micro-batches, oldest first)."""
        import numpy as np
        st = ServeStats()
        rec = np.zeros(max_records, np.dtype(BATCH_RECORD_DTYPE))
        n = ctypes.c_int32()
        _check("hough_serve_trace", load().hough_serve_trace(self.handle, ctypes.byref(st),
                                                             ctypes.c_void_p(rec.ctypes.data), max_records,
                                                             ctypes.byref(n)))
        stall = lambda w: {k: int(getattr(w, k)) for k, _ in ServeStall._fields_}  # noqa: E731
        return ({"passes": int(st.passes), "batches": int(st.batches), "stall_ns": int(st.stall_ns),
                 "loop": stall(st.loop), "submit": stall(st.submit)}, rec[: n.value])

    def inject_launch_failures(self, n: int):
        """Test hook: the next n micro-batch launches fail on the host before anything is enqueued."""
        _check("hough_serve_inject_launch_failures", load().hough_serve_inject_launch_failures(self.handle, int(n)))

    def close(self):
        if self.handle:
            rc = load().hough_serve_close(self.handle)
            self.handle = ctypes.c_void_p()
            _check("hough_serve_close", rc)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def set_host_timing(on: bool):
    """Per-stage CUDA-event timing of later HostRunner calls on this thread (HostRunner.stage_ms)."""
    load().hough_set_host_timing(1 if on else 0)


def set_stage_events(begin=None, end=None):
    """Records torch.cuda.Event pairs around the fused kernel of later calls on this thread."""
    load().hough_set_stage_events(ctypes.c_void_p(begin.cuda_event) if begin is not None else None,
                                  ctypes.c_void_p(end.cuda_event) if end is not None else None)


def autotune(xy, off, p: Params, stream=None):
    """Fastest launch shape for p on this sample batch (device tensors): (tuned Params, ms or -1 if cached)."""
    torch = _torch()
    xy = _dev(xy, "xy", torch.int32)
    off = _dev(off, "off", torch.int64)
    q = Params(*[getattr(p, n) for n, _ in Params._fields_])
    lib = load()
    nb = int(lib.hough_autotune_scratch_size(ctypes.byref(q), xy.shape[0], off.shape[0] - 1))
    scratch = torch.empty(nb, dtype=torch.uint8, device=xy.device)
    st = new_status(xy.device)
    ms = ctypes.c_float()
    _check("hough_autotune", lib.hough_autotune(ctypes.byref(q), _ptr(xy), xy.shape[0], _ptr(off), off.shape[0] - 1,
                                                _ptr(scratch), nb, _ptr(st), _stream(stream), ctypes.byref(ms)))
    return q, float(ms.value)


def selftest_bin(n_rho: int, rho_lo: int, rho_hi: int, stream=None) -> int:
    torch = _torch()
    mism = torch.zeros(1, dtype=torch.int64, device="cuda")
    _check("hough_selftest_bin", load().hough_selftest_bin(n_rho, rho_lo, rho_hi, _ptr(mism), _stream(stream)))
    return mism


def selftest_fpbin(n_theta: int, n_rho: int, seed: int, n_samples: int, stream=None):
    """(disagreements, exact-path fallbacks) of the vote's general float bin path, then
    (disagreements, exact-path fallbacks, samples) of the mirror-pair bit-pattern row, on
    random tuples."""
    torch = _torch()
    out = torch.zeros(5, dtype=torch.int64, device="cuda")
    _check("hough_selftest_fpbin", load().hough_selftest_fpbin(n_theta, n_rho, seed, n_samples, _ptr(out),
                                                               _stream(stream)))
    return tuple(int(x) for x in out.tolist())


def phase_cycles(reset: bool = True):
    """(enabled, {phase: cycles}) of the fused kernel's phase counters since the last reset
    (thread 0 of every CTA, summed). enabled is False unless the library is the phase-timer
    build (HOUGH_PHASE_TIMERS=1 in the environment before the first load); the counts are
    then 0. Synchronises the device."""
    buf = (ctypes.c_uint64 * len(PHASES))()
    en = ctypes.c_int32(0)
    _check("hough_phase_cycles", load().hough_phase_cycles(buf, len(PHASES), 1 if reset else 0, ctypes.byref(en)))
    return bool(en.value), {name: int(buf[i]) for i, name in enumerate(PHASES)}


def probe_smem_atomics(mode: int, ctas_per_sm: int, threads: int, smem_bytes: int, iters: int, sink, stream=None):
    _check("hough_probe_smem_atomics", load().hough_probe_smem_atomics(mode, ctas_per_sm, threads, smem_bytes, iters,
                                                                       _ptr(sink), _stream(stream)))
