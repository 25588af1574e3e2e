"""Benchmark of the conformal Hough hit filter on GB300.

One step = the whole hot path (validate/order, map, rho, vote, peaks, select) over
one batch of synthetic events resident in HBM, launched through the C ABI
(``hough_run_batched``: persistent work-queue kernel replayed as a CUDA graph).
Prints one JSON line. ``--impl reference`` times the CPU oracle instead.

Multi-GPU (torchrun): every rank processes its own batch of the same size (weak
scaling, no collective on the data path); the timed region is bracketed by
barriers and the max over ranks is reported.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gen  # noqa: E402

METRIC = "events/s and p99 event latency on 1 GB300 (batched/served vs plain), bit-exact"
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "fused_kernel_batched_traffic.txt")
PEAK_RECORD_BYTES = 8
KERNEL_SOURCES = ["paper_2607_04067_gb300/csrc/hough_fused.cu", "paper_2607_04067_gb300/csrc/hough_device.cuh"]


def kernel_hash() -> str:
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return ws, int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0"))


def shard_first_event(rank: int, events_per_rank: int) -> int:
    """Weak scaling: rank r owns events [r n, (r + 1) n) of the workload's seeded event stream."""
    return rank * events_per_rank


def max_over_ranks(x: float, dist, device) -> float:
    """The largest x over all ranks (the job's time is its slowest rank's); x itself alone."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """Samples SM clock and throttle reasons with nvidia-smi while the timed region runs."""

    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.lines = []
        self.t = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.t:
                self.t.join(timeout=2)

    def summary(self):
        mhz, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            if self.uuid and self.uuid not in f[0]:
                continue
            try:
                mhz.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not mhz:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(mhz)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(mhz)}


T0 = time.perf_counter()


def progress(what: str):
    """Elapsed wall time of the run on stderr (the JSON line stays the only stdout line)."""
    print(f"[bench {time.perf_counter() - T0:7.1f} s] {what}", file=sys.stderr, flush=True)


def workload_config(cfg, n_events, args):
    """The workload a line is measured on: identical in the GPU arm and the reference arm."""
    return {"workload": cfg.name, "events_per_gpu": n_events, "n_theta": cfg.n_theta, "n_rho": cfg.n_rho,
            "threshold": cfg.threshold, "keep_halfwidth": cfg.keep_halfwidth, "max_peaks": cfg.max_peaks,
            "peak_finder": peak_finder_name(args), "parallelism": "events sharded over ranks, no collective"}


def peak_args(args):
    """(peak_mode, rel_num, rel_den, nms_radius) of the command line."""
    if getattr(args, "peak_mode", "local-max") != "iterative":
        return 0, 0, 1, 1
    num, den = (int(x) for x in args.rel.split("/"))
    return 1, num, den, args.nms_radius


def peak_finder_name(args) -> str:
    if getattr(args, "peak_mode", "local-max") != "iterative":
        return "3x3 local maxima"
    return f"iterative, relative threshold {args.rel} of the maximum, suppression radius {args.nms_radius}"


def oracle_baseline(cfg, ev, budget_events: int, threads: int, peak=(0, 0, 1, 1)):
    """The CPU oracle as it stands, timed on the host cores over the first events of the batch."""
    import oracle
    n = min(budget_events, ev.n_events)
    off = ev.off[: n + 1]
    xy = ev.xy[: int(off[-1])]
    p = oracle.params(cfg.n_theta, cfg.n_rho, cfg.threshold, cfg.keep_halfwidth, cfg.max_peaks, *peak)
    t0 = time.perf_counter()
    r = oracle.run(xy, off, p, threads=threads)
    dt = time.perf_counter() - t0
    return n / dt, r, n, dt


def sized_sample(cfg, ev, want: int, threads: int, peak, seconds: float) -> int:
    """Events of a CPU sample of about `seconds` (at most `want`), sized from a short probe run, so
    that slow oracle configurations (the iterative finder at 512 x 512) stay within a bounded time."""
    probe = min(want, max(32, 8 * threads))
    v, _, _, _ = oracle_baseline(cfg, ev, probe, threads, peak)
    return max(probe, min(want, int(v * seconds)))


def run_reference(args, cfg):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    per_step = args.ref_events
    ev = gen.generate(cfg, per_step, with_truth=False)
    for _ in range(max(0, args.warmup)):
        oracle_baseline(cfg, ev, per_step, threads, peak_args(args))
    times = []
    for _ in range(args.steps):
        _, _, n, dt = oracle_baseline(cfg, ev, per_step, threads, peak_args(args))
        times.append(dt)
    total = sum(times)
    value = per_step * args.steps / total
    sample = (f"{per_step} events of the {cfg.name} workload per step (the first events of its seeded batch), "
              f"timed on {threads} host threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": workload_config(cfg, args.events or cfg.n_events, args),
        "sample": {"events_per_step": per_step, "note": "the oracle times a bounded sample of the workload"},
        "cpu_baseline": {"value": value, "unit": "events/s", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def probe_atomic_ceiling(h, torch, stream):
    """Shared-memory red.add throughput (ops/s): lane-private banks and pseudo-random words."""
    out = {}
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for mode, name in ((0, "lane_bank"), (4, "lane_bank_random_rows"), (1, "random_word")):
        ctas, threads, smem, iters = 2, 1024, 96 * 1024, 400
        for _ in range(2):
            h.probe_smem_atomics(mode, ctas, threads, smem, iters, sink, stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        e0.record(stream)
        for _ in range(reps):
            h.probe_smem_atomics(mode, ctas, threads, smem, iters, sink, stream)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        ops = sms * ctas * threads * iters * 16
        out[name] = ops / (ms * 1e-3)
    return out


def serve_stream(h, p, kw, pool, arrival, max_batch_hits=1 << 22):
    """One arrival stream through a server configured by kw: sustained events/s (completed over
    the span from the first scheduled arrival to the last result), latency percentiles from
    scheduled arrival to results in host memory, device flags, and the loop's stall watch."""
    res = h.Server.result_array(len(arrival))  # written now: the loop faults in no pages
    with h.Server(p, max_batch_hits=max_batch_hits, queue_capacity=1 << 16, **kw) as srv:
        t0 = srv.replay(pool.xy, pool.off, arrival, results_out=res)
        srv.drain(300)
        stats, rec = srv.trace()
    lat = (res["t_done_ns"] - res["t_arrival_ns"]) / 1e3
    span = (res["t_done_ns"].max() - t0) / 1e9 if len(res) else float("nan")
    out = {"sustained_events_per_s": len(res) / span, "p50_us": float(np.percentile(lat, 50)),
           "p99_us": float(np.percentile(lat, 99)), "p999_us": float(np.percentile(lat, 99.9)),
           "completed": int(len(res)), "flags": int(np.bitwise_or.reduce(res["status"])),
           "batches": stats["batches"], "mean_batch_events": float(rec["n_events"].mean()) if len(rec) else None,
           "stalls": {w: dict(stats[w], max_gap_at_ms=(stats[w]["max_gap_at"] - t0) / 1e6 if stats[w]["count"] else None)
                      for w in ("loop", "submit")}}
    if len(rec):  # where a micro-batch's time goes (medians over the stream's most recent batches)
        out["batch_us"] = {"gather_and_enqueue": float(np.median(rec["t_launched"] - rec["t_gather"]) / 1e3),
                           "device_and_copies": float(np.median(rec["t_done_seen"] - rec["t_launched"]) / 1e3),
                           "results_to_callers": float(np.median(rec["t_finished"] - rec["t_done_seen"]) / 1e3)}
    return out


SERVED = dict(slots=4, max_batch_events=256, flush_us=50.0)
PLAIN_1000 = dict(slots=1, max_batch_events=1000, flush_us=0.0)


def measure_serving(h, cfg, p, rates, seconds, flush_us=50.0, pool_events=20000, seed=11, sat_events=300_000,
                    sat_rates=(1_000_000, 2_000_000, 4_000_000), sat_seconds=0.25):
    """Continuous-batching server (4 slots, micro-batches of at most 256 events, launched after
    flush_us) vs plain per-batch launches of 1,000 events (one batch in flight, launched when
    full), both fed the same Poisson arrival streams. Streams at the offered rates, streams past
    saturation, and a closed-loop run (every request arrives at t = 0: the loop's capacity).
    Latency runs from each event's scheduled arrival to its results in host memory."""
    pool = gen.generate(cfg, pool_events, with_truth=False)
    rng = np.random.default_rng(seed)
    served = dict(SERVED, flush_us=flush_us)
    arms = (("served", served), ("plain_1000", PLAIN_1000))
    streams = []
    for rate, secs in [(r, seconds) for r in rates] + [(r, sat_seconds) for r in sat_rates]:
        progress(f"serving stream {rate} events/s")
        n = int(rate * secs)
        arrival = np.cumsum(rng.exponential(1e9 / rate, size=n)).astype(np.int64)
        row = {"offered_events_per_s": rate, "seconds": secs, "events": n, "flush_us": flush_us}
        for name, kw in arms:
            row[name] = serve_stream(h, p, kw, pool, arrival)
        streams.append(row)
    closed = {}
    for name, kw in arms:
        if sat_events:
            closed[name] = serve_stream(h, p, kw, pool, np.zeros(sat_events, np.int64))
    # the highest offered rate whose p99 stays within 200 us, per arm
    best = {}
    for name, _ in arms:
        ok = [r["offered_events_per_s"] for r in streams if r[name]["p99_us"] <= 200.0 and
              r[name]["completed"] == r["events"]]
        best[name] = max(ok) if ok else None
    return {"streams": streams, "closed_loop": {"events": sat_events, **closed},
            "highest_offered_rate_with_p99_le_200us": best,
            "arms": {"served": served, "plain_1000": PLAIN_1000}}


PT_BINS = (50.0, 100.0, 200.0, 400.0, 800.0, 1500.0)


def track_finding(h, cfg, out, p, first_event: int, n_sample: int, dpt_max=20.0, dphi_max=0.05):
    """Eq. (2) circles of the stored peaks against the generator's true tracks on the first
    n_sample events: a track is found when some peak's circle has |pT - pT_true| < dpt_max MeV/c
    and its centre direction lies within dphi_max rad of the true one. Efficiency per pT bin, and
    the pT and direction residuals of the closest peak of each found track."""
    import torch
    n = min(n_sample, out.npeaks.shape[0])
    circ = h.circles(out.npeaks[:n], out.peaks[:n], p, 1.0).cpu().numpy()
    npk = np.minimum(out.npeaks[:n].cpu().numpy(), p.max_peaks)
    found = np.zeros(len(PT_BINS) - 1, np.int64)
    total = np.zeros(len(PT_BINS) - 1, np.int64)
    dpt, dphi = [], []
    for e in range(n):
        c = circ[e, : npk[e]]
        phic = np.arctan2(c[:, 1], c[:, 0])
        for pt, q, phi0 in gen.event_tracks(cfg, first_event + e):
            b = int(np.searchsorted(PT_BINS, pt, side="right")) - 1
            if b < 0 or b >= len(total):
                continue
            total[b] += 1
            if not len(c):
                continue
            d = np.angle(np.exp(1j * (phic - (phi0 - q * np.pi / 2))))
            ok = (np.abs(c[:, 3] - pt) < dpt_max) & (np.abs(d) < dphi_max)
            if ok.any():
                found[b] += 1
                i = int(np.argmin(np.where(ok, np.abs(c[:, 3] - pt) / dpt_max + np.abs(d) / dphi_max, np.inf)))
                dpt.append(c[i, 3] - pt)
                dphi.append(d[i])
    return {"events": n, "criterion": f"|dpT| < {dpt_max} MeV/c and |dphi_centre| < {dphi_max} rad",
            "efficiency_by_pt_mev": {f"{PT_BINS[i]:.0f}-{PT_BINS[i + 1]:.0f}":
                                     (float(found[i] / total[i]) if total[i] else None) for i in range(len(total))},
            "tracks": int(total.sum()), "found": int(found.sum()),
            "dpt_rms_mev": float(np.sqrt(np.mean(np.square(dpt)))) if dpt else None,
            "dphi_rms_mrad": float(1e3 * np.sqrt(np.mean(np.square(dphi)))) if dphi else None}


def compare_with_oracle(r, n, ev, out, max_peaks):
    """Outputs of the timed batch's first n events against the oracle's, element by element:
    peak counts, kept counts, stored peak records and the kept-hit masks."""
    npk = out.npeaks[:n].cpu().numpy()
    nk = out.nkept[:n].cpu().numpy()
    a = int(ev.off[n])
    mask = out.mask[:a].cpu().numpy()
    pk = np.ascontiguousarray(out.peaks[:n].cpu().numpy().astype(np.int16))
    bad = set(np.nonzero(npk != r.npeaks)[0].tolist()) | set(np.nonzero(nk != r.nkept)[0].tolist())
    diff = np.nonzero(mask != r.mask)[0]
    if len(diff):
        bad |= set((np.searchsorted(ev.off[: n + 1], diff, side="right") - 1).tolist())
    import oracle
    view = pk.view(oracle.PEAK_DTYPE).reshape(n, -1)
    for e in range(n):
        s = min(int(r.npeaks[e]), max_peaks)
        if e not in bad and not np.array_equal(view[e, :s], r.peaks[e, :s]):
            bad.add(e)
    return {"events": n, "hits": a, "mismatches": len(bad), "compared": "npeaks, nkept, peak records, kept mask",
            "first_bad_events": sorted(bad)[:5]}


def vote_phase_fraction(args, cfg, lane_bank, sms, sm_mhz):
    """The vote phase alone against the conflict-free atomic ceiling: the phase-timer build of the
    library (same results, clock64 marks) runs the workload's first 20,000 events in a child
    process; vote cycles per event on one SM give votes per SM-cycle, against the ceiling per
    SM-cycle at the clock sampled in the timed region."""
    cmd = [sys.executable, os.path.abspath(__file__), "--phase-split", "0", "--workload", cfg.name, "--events",
           str(min(20000, args.events or cfg.n_events))]
    if getattr(args, "peak_mode", "local-max") == "iterative":
        cmd += ["--peak-mode", "iterative", "--rel", args.rel, "--nms-radius", str(args.nms_radius)]
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=ROOT)
        d = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])
    except (subprocess.SubprocessError, IndexError, ValueError) as e:
        return {"unavailable": f"phase-timer run failed: {type(e).__name__}"}
    row = next(iter(d["rows"].values()))
    if "cycles_per_event" not in row:
        return {"unavailable": row.get("unavailable", "no phase counters")}
    cyc = row["cycles_per_event"]
    votes_per_event = d["hits"] * cfg.n_theta / d["events"]
    mhz = sm_mhz or 2070.0
    ceil_per_sm_cycle = lane_bank / (sms * mhz * 1e6)
    per_cycle = votes_per_event / cyc["vote"]
    return {"vote_cycles_per_event": cyc["vote"], "event_cycles": sum(cyc.values()), "block": row.get("block"),
            "votes_per_sm_cycle": per_cycle, "ceiling_per_sm_cycle": ceil_per_sm_cycle,
            "frac": per_cycle / ceil_per_sm_cycle, "events": d["events"],
            "basis": "phase-timer build, thread 0 clock64 between the barriers around the vote"}


def run_phase_split(args, cfg):
    """Cycles per event of each phase of the fused kernel against CTA size (the paper's
    per-stage study, Sec. 4). The phase-timer build of the library (HOUGH_PHASE_TIMERS, same
    results) runs the batched launch of the workload's first events once per block size after
    warm-up; thread 0 of every CTA adds the clock64() cycles of each phase of its items. One
    JSON line: per block size, cycles per event by phase (summed over the CTAs, divided by
    the events) and the events/s of that instrumented launch."""
    os.environ["HOUGH_PHASE_TIMERS"] = "1"
    import torch
    import paper_2607_04067_gb300 as h

    torch.cuda.set_device(0)
    n = args.events or min(cfg.n_events, 20000)
    ev = gen.generate(cfg, n, with_truth=False)
    xy, off = torch.from_numpy(ev.xy).cuda(), torch.from_numpy(ev.off).cuda()
    stream = torch.cuda.Stream()
    rows, peak = {}, peak_args(args)
    for blk in (int(x) for x in args.phase_split.split(",")):
        p = None
        for tiles in (1, 0):  # one tile where the accumulator fits one CTA (block 0: the plan's)
            q = h.params(cfg.n_theta, cfg.n_rho, cfg.threshold, cfg.keep_halfwidth, cfg.max_peaks, theta_tiles=tiles,
                         block=blk, events_per_cta=1)
            q.peak_mode, q.rel_num, q.rel_den, q.nms_radius = peak
            try:
                h.resolve(q)
                p = q
                break
            except h.HoughError:
                continue
        if p is None:
            rows[str(blk)] = {"unavailable": "no plan with this block size"}
            continue
        out = h.alloc_outputs(ev.n_hits, n, p)
        with torch.cuda.stream(stream):
            for _ in range(3):
                h.run(xy, off, p, out=out, batched=True, stream=stream)
        stream.synchronize()
        h.phase_cycles(reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            h.run(xy, off, p, out=out, batched=True, stream=stream)
            e1.record(stream)
        e1.synchronize()
        enabled, cyc = h.phase_cycles(reset=True)
        if not enabled:
            raise RuntimeError("the library loaded is not the phase-timer build")
        if h.status(out.status, stream) != 0:
            raise RuntimeError("device status flags set")
        r = h.resolve(p)
        rows[str(blk)] = {"theta_tiles": r.theta_tiles, "block": r.block, "events_per_s": n / (e0.elapsed_time(e1) * 1e-3),
                          "cycles_per_event": {k: round(v / n) for k, v in cyc.items() if v}}
    print(json.dumps({"metric": "fused-kernel cycles per event by phase (thread 0 of each CTA)",
                      "workload": cfg.name, "events": n, "hits": ev.n_hits, "n_theta": cfg.n_theta,
                      "n_rho": cfg.n_rho, "peak_finder": args.peak_mode, "build": "phase timers",
                      "rows": rows}))
    return 0


def run_sweep(args, cfg):
    """Batch-size sweep on one GPU (the paper's runtime-versus-event-count study, Sec. 4): for
    each batch of the workload's first n events, events/s of the batched launch (persistent
    kernel in a CUDA graph), of the plain launch (one CTA per event) and of the stepwise path
    with its per-stage times (accumulator through HBM), events/s of the batched launch per CTA
    size, and the CPU oracle on the host cores. One JSON line per batch size."""
    import torch
    import paper_2607_04067_gb300 as h

    torch.cuda.set_device(0)
    sizes = [int(x) for x in args.sweep.split(",")]
    full = gen.generate(cfg, max(sizes), with_truth=False)
    base = h.params(cfg.n_theta, cfg.n_rho, cfg.threshold, cfg.keep_halfwidth, cfg.max_peaks)
    stream = torch.cuda.Stream()
    threads = os.cpu_count() or 1

    def timed(fn, reps):
        with torch.cuda.stream(stream):
            for _ in range(3):
                fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    for n in sizes:
        off_np = full.off[: n + 1]
        xy = torch.from_numpy(full.xy[: int(off_np[-1])]).cuda()
        off = torch.from_numpy(off_np).cuda()
        reps = max(3, min(200, 200000 // max(n, 1)))
        row = {"workload": cfg.name, "events": n, "hits": int(off_np[-1])}
        out = h.alloc_outputs(xy.shape[0], n, base)
        row["batched_events_per_s"] = n / (timed(lambda: h.run(xy, off, base, out=out, batched=True,
                                                                stream=stream), reps) * 1e-3)
        row["plain_events_per_s"] = n / (timed(lambda: h.run(xy, off, base, out=out, stream=stream), reps) * 1e-3)
        per_block = {}
        for blk in (256, 512, 1024):
            q = h.params(cfg.n_theta, cfg.n_rho, cfg.threshold, cfg.keep_halfwidth, cfg.max_peaks, theta_tiles=1,
                         block=blk, events_per_cta=1)
            try:
                oq = h.alloc_outputs(xy.shape[0], n, q)
                per_block[str(blk)] = n / (timed(lambda: h.run(xy, off, q, out=oq, batched=True, stream=stream),
                                                 reps) * 1e-3)
            except h.HoughError:
                per_block[str(blk)] = None
        row["batched_events_per_s_by_block"] = per_block
        if n <= args.sweep_stepwise_max:
            st = h.new_status()
            uq = torch.empty(xy.shape[0], dtype=torch.int64, device="cuda")
            vq = torch.empty_like(uq)
            acc = torch.empty((n, cfg.n_theta, cfg.n_rho), dtype=torch.int16, device="cuda")
            npk, pk = h.peaks(acc, base, st, stream=stream)  # allocates the peak buffers once
            mask = torch.empty(xy.shape[0], dtype=torch.uint8, device="cuda")
            nk = torch.empty(n, dtype=torch.int32, device="cuda")
            stages = {
                "map": lambda: h.map_hits(xy, off, st, uq, vq, stream=stream),
                "vote": lambda: h.vote(uq, vq, off, base, st, acc, stream=stream),
                "peaks": lambda: h.peaks(acc, base, st, npk, pk, stream=stream),
                "select": lambda: h.select(uq, vq, off, base, npk, pk, st, mask, nk, stream=stream),
            }
            ms = {k: timed(f, max(3, reps // 4)) for k, f in stages.items()}
            row["stepwise_stage_ms"] = ms
            row["stepwise_events_per_s"] = n / (sum(ms.values()) * 1e-3)
        if n <= args.sweep_oracle_max:
            v, _, _, _ = oracle_baseline(cfg, full, n, threads)
            row["oracle_events_per_s"] = v
            row["oracle_threads"] = threads
        print(json.dumps(row), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched", choices=sorted(gen.CONFIGS))
    ap.add_argument("--events", type=int, default=0, help="events per rank (0 = the workload's size)")
    ap.add_argument("--ref-events", type=int, default=3000, help="oracle events per reference step")
    ap.add_argument("--cpu-sample", type=int, default=10000,
                    help="most oracle events for cpu_baseline and parity (sized to ~20 s; ~15 s on one thread)")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle baseline (profiling runs)")
    ap.add_argument("--serve-seconds", type=float, default=2.0, help="length of each serving stream")
    ap.add_argument("--serve-flush-us", type=float, default=50.0,
                    help="serving loop: longest wait of a request before its partial micro-batch is launched")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-phase", action="store_true", help="skip the vote-phase fraction (phase-timer child run)")
    ap.add_argument("--serve-only", type=int, default=0,
                    help="only the serving streams, this many times over (stall study); one JSON line per repeat")
    ap.add_argument("--no-tune", action="store_true", help="use the default launch shape instead of the autotuner")
    ap.add_argument("--tune-events", type=int, default=10000, help="events of the batch the autotuner times")
    ap.add_argument("--shape", default="", help="fixed launch shape 'theta_tiles,block,events_per_cta' (profiling)")
    ap.add_argument("--peak-mode", default="local-max", choices=["local-max", "iterative"],
                    help="peak finder: one-pass 3x3 local maxima, or the paper's iterative finder")
    ap.add_argument("--rel", default="1/2", help="iterative finder: relative threshold as a fraction of the maximum")
    ap.add_argument("--nms-radius", type=int, default=3, help="iterative finder: suppression half-width in bins")
    ap.add_argument("--physics-events", type=int, default=2000,
                    help="events whose peaks are matched to the true tracks (Eq. 2 circles)")
    ap.add_argument("--sweep", default="", help="batch-size sweep instead of the benchmark, e.g. '1,10,100,1000'")
    ap.add_argument("--sweep-stepwise-max", type=int, default=10000, help="largest batch run through the stepwise path")
    ap.add_argument("--sweep-oracle-max", type=int, default=10000, help="largest batch timed on the CPU oracle")
    ap.add_argument("--phase-split", default="",
                    help="per-phase cycles of the fused kernel for these block sizes, e.g. '256,512,1024'")
    args = ap.parse_args()
    cfg = gen.CONFIGS[args.workload]
    if args.impl == "reference":
        return run_reference(args, cfg)
    if args.sweep:
        return run_sweep(args, cfg)
    if args.phase_split:
        return run_phase_split(args, cfg)
    if args.serve_only:
        import torch
        import paper_2607_04067_gb300 as h
        torch.cuda.set_device(0)
        scfg = gen.CONFIGS["served"]
        sp = h.params(scfg.n_theta, scfg.n_rho, scfg.threshold, scfg.keep_halfwidth, scfg.max_peaks)
        for rep in range(args.serve_only):
            res = measure_serving(h, scfg, sp, (50_000, 200_000, 400_000), args.serve_seconds, args.serve_flush_us,
                                  seed=11 + rep, sat_rates=(), sat_events=0)
            print(json.dumps({"metric": "served streams", "repeat": rep, **res}), flush=True)
        return 0

    import torch
    import paper_2607_04067_gb300 as h

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    n_events = args.events or cfg.n_events
    ev = gen.generate(cfg, n_events, first_event=shard_first_event(rank, n_events), with_truth=(rank == 0))
    xy = torch.from_numpy(ev.xy).cuda()
    off = torch.from_numpy(ev.off).cuda()
    p = h.params(cfg.n_theta, cfg.n_rho, cfg.threshold, cfg.keep_halfwidth, cfg.max_peaks)
    p.peak_mode, p.rel_num, p.rel_den, p.nms_radius = peak_args(args)
    tune_ms = None
    if args.shape:
        p.theta_tiles, p.block, p.events_per_cta = (int(x) for x in args.shape.split(","))
    elif not args.no_tune:
        ns = min(n_events, args.tune_events)
        p, tune_ms = h.autotune(xy[: int(ev.off[ns])], off[: ns + 1], p)
    plan = h.resolve(p)
    out = h.alloc_outputs(ev.n_hits, ev.n_events, p)
    stream = torch.cuda.Stream()
    pairs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(2)]
    for b_, e_ in pairs:  # torch only reports elapsed time for events it has recorded once itself;
        b_.record(stream)  # later records of the same native events are made by the library
        e_.record(stream)

    def step(i):
        h.set_stage_events(*pairs[i % 2])
        h.run(xy, off, p, out=out, batched=True, stream=stream)

    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for i in range(max(args.warmup, 3)):
            step(i)
    stream.synchronize()
    flags = h.status(out.status, stream)

    progress("warm-up done")
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kern_ms = []
    barrier()
    with ClockSampler(uuid) as clocks:
        with torch.cuda.stream(stream):
            t_start.record(stream)
            for i in range(args.steps):
                step(i)
                if i >= 1:
                    b, e = pairs[(i - 1) % 2]
                    e.synchronize()
                    kern_ms.append(b.elapsed_time(e))
            t_end.record(stream)
        t_end.synchronize()
        b, e = pairs[(args.steps - 1) % 2]
        kern_ms.append(b.elapsed_time(e))
    barrier()
    h.set_stage_events(None, None)
    elapsed = max_over_ranks(t_start.elapsed_time(t_end), dist, "cuda")
    ms_step = elapsed / args.steps
    total_events = n_events * ws * args.steps
    value = total_events / (elapsed * 1e-3)

    progress("timed steps done")
    # end to end through the host-buffer entry point (pinned host in, host results out)
    xy_h = torch.from_numpy(ev.xy).pin_memory()
    off_h = torch.from_numpy(ev.off).pin_memory()
    stored = int(out.npeaks.clamp(max=cfg.max_peaks).sum().item())
    runner = h.HostRunner(ev.n_hits, ev.n_events, p, peaks_cap=stored + stored // 8 + 1024)
    for _ in range(2):  # graphs, streams and host pages warm
        runner(xy_h, off_h, stream)
    barrier()
    call_ms = []
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        t1 = time.perf_counter()
        runner(xy_h, off_h, stream)
        call_ms.append(1e3 * (time.perf_counter() - t1))
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e_value = n_events * ws * args.e2e_steps / e2e_s
    h2d = ev.xy.nbytes + ev.off.nbytes
    d2h = runner.d2h_bytes()
    # one more call, outside the timed region, with CUDA-event marks around every stage
    h.set_host_timing(True)
    t1 = time.perf_counter()
    runner(xy_h, off_h, stream)
    e2e_stages = dict(runner.stage_ms(), call_wall=1e3 * (time.perf_counter() - t1))
    h.set_host_timing(False)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    progress("end to end done")
    peaks_meas, peaks_kind = measured_peaks()
    votes = ev.n_hits * cfg.n_theta
    kern = float(np.mean(kern_ms))
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    traffic = None
    try:
        with open(PROFILE_TRAFFIC) as f:
            kv = dict(line.split(":", 1) for line in f if ":" in line and not line.startswith("#"))
        if kv.get("kernel_sha256_16", "").strip() == kernel_hash() and \
                kv.get("workload", "").strip() == cfg.name and int(kv.get("events", "0")) == n_events:
            traffic = float(kv["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        traffic = None
    ceiling = probe_atomic_ceiling(h, torch, stream)
    votes_per_s = votes / (kern * 1e-3)
    npk = out.npeaks.cpu().numpy()
    stored = int(np.minimum(npk, cfg.max_peaks).sum())
    # algorithmic HBM bytes of one launch: hits in (8 B) and kept flags out (1 B), per event its
    # offsets (8 B), peak count and kept count (4 B each), and the stored peak records (8 B each)
    hbm_bytes = ev.n_hits * 9 + n_events * 16 + stored * PEAK_RECORD_BYTES
    clk = clocks.summary()

    # parity of the timed batch itself: its first events (up to --cpu-sample, about 20 s of the
    # oracle on the host threads) against the oracle
    cpu = parity = None
    if not args.no_cpu:
        threads = os.cpu_count() or 1
        n_par = sized_sample(cfg, ev, args.cpu_sample, threads, peak_args(args), 20.0)
        v, r, n, dt = oracle_baseline(cfg, ev, n_par, threads, peak_args(args))
        parity = compare_with_oracle(r, n, ev, out, cfg.max_peaks)
        n_one = max(1, min(n // 10, int(v / threads * 15.0)))  # about 15 s on one thread
        v1, _, n1, dt1 = oracle_baseline(cfg, ev, n_one, 1, peak_args(args))
        cpu = {"value": v, "unit": "events/s", "cores": threads, "kind": "oracle",
               "sample": f"first {n} events of this batch ({dt:.1f} s wall on {threads} threads, events in parallel)",
               "single_thread": {"value": v1, "unit": "events/s", "cores": 1,
                                 "sample": f"first {n1} events of this batch ({dt1:.1f} s on 1 thread)"}}

    progress("oracle and parity done")
    vote_phase = None
    if not args.no_phase:
        vote_phase = vote_phase_fraction(args, cfg, ceiling["lane_bank"], sms, clk.get("sm_mhz"))

    progress("vote phase done")
    served = None
    if not args.no_serve:
        scfg = gen.CONFIGS["served"]
        served = measure_serving(h, scfg, h.params(scfg.n_theta, scfg.n_rho, scfg.threshold, scfg.keep_halfwidth,
                                                   scfg.max_peaks), (50_000, 200_000, 400_000), args.serve_seconds,
                                 args.serve_flush_us)

    progress("serving done")
    import oracle
    rc, rs = oracle.metrics(out.mask.cpu().numpy(), ev.truth) if ev.truth is not None else (None, None)
    lane = ceiling["lane_bank"]
    line = {
        "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": workload_config(cfg, n_events, args),
        "launch": {"theta_tiles": plan.theta_tiles, "block": plan.block, "events_per_cta": plan.events_per_cta,
                   "autotuned": not (args.no_tune or args.shape), "tune_best_ms": tune_ms,
                   "path": "hough_run_batched (persistent kernel + CUDA graph)",
                   "l2": f"inputs {ev.xy.nbytes / 1e9:.2f} GB > 129 MB L2, no flush", "hits_per_gpu": ev.n_hits},
        "hits_per_s": ev.n_hits * ws * args.steps / (elapsed * 1e-3),
        "parity": parity,
        "latency": {"batch_ms": ms_step, "note": "every event of the batch completes within one step"},
        "served": served,
        "e2e": {"value": e2e_value, "unit": "events/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "stages_ms": e2e_stages, "calls_ms": [round(x, 2) for x in call_ms]},
        "gpu_launches": 2 * args.steps,
        "roofline": {"bound": "smem_atomic", "kernel": "fused_kernel (persistent)",
                     "achieved": votes_per_s / 1e9, "peak": lane / 1e9, "unit": "Gvotes/s",
                     "frac": votes_per_s / lane, "traffic": traffic,
                     "peak_basis": "measured red.shared.add.u32 throughput, every lane of a warp on its own bank "
                                   "(hough_probe_smem_atomics mode 0, 2 CTAs x 1024 threads per SM), timed in this run",
                     "votes_per_launch": votes, "kernel_ms": kern, "votes_per_s": votes_per_s,
                     "lane_bank_random_rows_ceiling_votes_per_s": ceiling["lane_bank_random_rows"],
                     "random_word_ceiling_votes_per_s": ceiling["random_word"],
                     "frac_of_random_word": votes_per_s / ceiling["random_word"],
                     "vote_phase": vote_phase,
                     "hbm": {"algorithmic_bytes": hbm_bytes, "achieved_gbs": hbm_bytes / (kern * 1e-3) / 1e9,
                             "peak_gbs": peaks_meas["hbm_gbs"], "peak_kind": peaks_kind,
                             "frac": hbm_bytes / (kern * 1e-3) / (peaks_meas["hbm_gbs"] * 1e9)}},
        "clocks": clk,
        "status_flags": flags,
        "physics": {"R_c": rc, "R_s": rs, "mean_peaks_per_event": float(npk.mean()),
                    "note": "at the workload's absolute threshold the filter keeps almost every hit: "
                            "selection work is sized by the noise peaks",
                    "track_finding": track_finding(h, cfg, out, p, 0, args.physics_events)},
        "cpu_baseline": cpu,
    }
    progress("physics done")
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    if parity is not None and parity["mismatches"]:
        sys.exit(3)


if __name__ == "__main__":
    main()
