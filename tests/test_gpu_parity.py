"""GPU parity: the CUDA path through the C ABI against the CPU oracle, element by element.

Integer path, so the bar is bit-exact equality of accumulators, peak lists, masks,
kept counts and accumulator checksums.
"""
import os

import numpy as np
import pytest

import gen
import oracle
from parity_util import assert_event_outputs_equal, peaks_np, sub_batch, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

THREADS = max(1, os.cpu_count() or 1)


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_04067_gb300 as hough
    hough.load()
    return hough


def cfg_params(h, cfg, **kw):
    return h.params(cfg.n_theta, cfg.n_rho, cfg.threshold, cfg.keep_halfwidth, cfg.max_peaks, **kw)


def dev(ev):
    return torch.from_numpy(ev.xy).cuda(), torch.from_numpy(ev.off).cuda()


def oracle_of(cfg, ev, with_acc=False, max_peaks=None, **kw):
    p = oracle.params(kw.get("n_theta", cfg.n_theta), kw.get("n_rho", cfg.n_rho), kw.get("threshold", cfg.threshold),
                      kw.get("keep_halfwidth", cfg.keep_halfwidth), max_peaks or cfg.max_peaks)
    return oracle.run(ev.xy, ev.off, p, with_acc=with_acc, threads=THREADS)


# ---------------------------------------------------------------- stepwise path

def test_stepwise_matches_oracle(h):
    cfg = gen.CONFIGS["plain_small"]
    ev = gen.generate(cfg)
    ref = oracle_of(cfg, ev, with_acc=True)
    xy, off = dev(ev)
    p = cfg_params(h, cfg)
    st = h.new_status()
    uq, vq = h.map_hits(xy, off, st)
    exp_u = np.array([oracle.map_hit(x, y)[1] for x, y in ev.xy[:2000]])
    exp_v = np.array([oracle.map_hit(x, y)[2] for x, y in ev.xy[:2000]])
    assert np.array_equal(to_np(uq)[:2000], exp_u) and np.array_equal(to_np(vq)[:2000], exp_v)
    acc = h.vote(uq, vq, off, p, st)
    assert np.array_equal(to_np(acc), ref.acc)
    npk, pk = h.peaks(acc, p, st)
    mask, nkept = h.select(uq, vq, off, p, npk, pk, st)
    assert h.status(st) == 0
    assert_event_outputs_equal(ref, npk, pk, mask, nkept, ev.off)


def test_stepwise_vote_tiled_large_accumulator(h):
    cfg = gen.CONFIGS["stress"]
    ev = gen.generate(cfg, 6)
    ref = oracle_of(cfg, ev, with_acc=True)
    xy, off = dev(ev)
    p = cfg_params(h, cfg)
    st = h.new_status()
    uq, vq = h.map_hits(xy, off, st)
    acc = h.vote(uq, vq, off, p, st)
    assert np.array_equal(to_np(acc), ref.acc)
    npk, pk = h.peaks(acc, p, st)
    mask, nkept = h.select(uq, vq, off, p, npk, pk, st)
    assert h.status(st) == 0
    assert_event_outputs_equal(ref, npk, pk, mask, nkept, ev.off)


# ---------------------------------------------------------------- fused path

@pytest.mark.parametrize("name,n", [("plain_small", None), ("plain_paper", None), ("batched", 400), ("stress", 24),
                                    ("paper_1000", 200)])
@pytest.mark.parametrize("batched", [False, True])
def test_fused_matches_oracle(h, name, n, batched):
    cfg = gen.CONFIGS[name]
    ev = gen.generate(cfg, n)
    ref = oracle_of(cfg, ev)
    xy, off = dev(ev)
    out = h.run(xy, off, cfg_params(h, cfg), checksum=True, batched=batched)
    assert h.status(out.status) == 0
    assert_event_outputs_equal(ref, out.npeaks, out.peaks, out.mask, out.nkept, ev.off, checksum=out.checksum)


@pytest.mark.parametrize("n_theta,n_rho,tiles,block", [
    (256, 256, 2, 0), (256, 256, 4, 0), (256, 256, 8, 0), (256, 256, 1, 256), (256, 256, 1, 1024),
    (256, 256, 3, 0), (64, 64, 2, 0), (64, 64, 1, 64), (100, 63, 1, 0), (100, 63, 3, 0), (4, 4, 1, 0),
    (1024, 1024, 0, 0), (1000, 1000, 0, 0), (37, 257, 2, 0),
    (512, 512, 4, 0), (512, 512, 8, 0), (128, 64, 2, 0), (128, 63, 2, 0)])
def test_shapes_and_tiles(h, n_theta, n_rho, tiles, block):
    cfg = gen.CONFIGS["plain_paper"]
    ev = gen.generate(cfg, 40)
    thr = max(2, cfg.threshold * min(n_theta, n_rho) // 256)
    ref = oracle.run(ev.xy, ev.off, oracle.params(n_theta, n_rho, thr, 1, 4096), threads=THREADS)
    xy, off = dev(ev)
    for batched in (False, True):
        out = h.run(xy, off, h.params(n_theta, n_rho, thr, 1, 4096, theta_tiles=tiles, block=block), checksum=True,
                    batched=batched)
        assert h.status(out.status) == 0
        assert_event_outputs_equal(ref, out.npeaks, out.peaks, out.mask, out.nkept, ev.off, checksum=out.checksum)


def test_checksum_off_gives_same_results(h):
    cfg = gen.CONFIGS["plain_paper"]
    ev = gen.generate(cfg, 50)
    xy, off = dev(ev)
    a = h.run(xy, off, cfg_params(h, cfg), checksum=True, batched=True)
    b = h.run(xy, off, cfg_params(h, cfg), checksum=False, batched=True)
    assert torch.equal(a.mask, b.mask) and torch.equal(a.npeaks, b.npeaks) and torch.equal(a.nkept, b.nkept)
    assert np.array_equal(peaks_np(a.peaks), peaks_np(b.peaks))


# ---------------------------------------------------------------- full-size workloads, sampled

@pytest.mark.parametrize("name,sample", [("batched", 300), ("stress", 60), ("paper_1000", 100)])
def test_full_size_sampled(h, name, sample):
    """Whole workload in the launch configuration the benchmark times (batched, no checksum),
    then the oracle recomputes a random sample of events one by one."""
    cfg = gen.CONFIGS[name]
    ev = gen.generate(cfg, with_truth=False)
    xy, off = dev(ev)
    p = cfg_params(h, cfg)
    out = h.run(xy, off, p, checksum=False, batched=True)
    assert h.status(out.status) == 0
    rng = np.random.default_rng(1)
    events = np.sort(rng.choice(ev.n_events, size=sample, replace=False))
    events[0] = 0
    events[-1] = ev.n_events - 1
    sxy, soff = sub_batch(ev.xy, ev.off, events)
    ref = oracle.run(sxy, soff, oracle.params(cfg.n_theta, cfg.n_rho, cfg.threshold, cfg.keep_halfwidth,
                                              cfg.max_peaks), threads=THREADS)
    assert_event_outputs_equal(ref, out.npeaks, out.peaks, out.mask, out.nkept, ev.off, events=events)
    # properties over every event
    nk = to_np(out.nkept)
    m = to_np(out.mask)
    csum = np.concatenate([[0], np.cumsum(m.astype(np.int64))])
    assert np.array_equal(csum[ev.off[1:]] - csum[ev.off[:-1]], nk)
    assert np.all(to_np(out.npeaks) <= cfg.max_peaks)
    assert set(np.unique(m)) <= {0, 1}
    # the shape the benchmark times: tuned on the first 10,000 events, whole batch again
    ns = min(ev.n_events, 10000)
    pt, _ = h.autotune(xy[: int(ev.off[ns])], off[: ns + 1], p)
    out2 = h.run(xy, off, pt, checksum=False, batched=True)
    assert h.status(out2.status) == 0
    assert torch.equal(out2.npeaks, out.npeaks) and torch.equal(out2.nkept, out.nkept)
    assert torch.equal(out2.mask, out.mask) and torch.equal(out2.peaks, out.peaks)


def test_full_size_sampled_iterative(h):
    """The batched workload (100,000 events) with the paper's iterative finder in the
    benchmark's configuration (half the maximum, radius 3, autotuned shape); the oracle
    recomputes a random sample of events one by one."""
    cfg = gen.CONFIGS["batched"]
    ev = gen.generate(cfg, with_truth=False)
    xy, off = dev(ev)
    kw = dict(peak_mode=1, rel_num=1, rel_den=2, nms_radius=3)
    p = cfg_params(h, cfg, **kw)
    p, _ = h.autotune(xy[: int(ev.off[10000])], off[:10001], p)
    out = h.run(xy, off, p, checksum=False, batched=True)
    assert h.status(out.status) == 0
    rng = np.random.default_rng(2)
    events = np.sort(rng.choice(ev.n_events, size=120, replace=False))
    events[0] = 0
    events[-1] = ev.n_events - 1
    sxy, soff = sub_batch(ev.xy, ev.off, events)
    ref = oracle.run(sxy, soff, oracle.params(cfg.n_theta, cfg.n_rho, cfg.threshold, cfg.keep_halfwidth,
                                              cfg.max_peaks, **kw), threads=THREADS)
    assert_event_outputs_equal(ref, out.npeaks, out.peaks, out.mask, out.nkept, ev.off, events=events)


# ---------------------------------------------------------------- edge cases

def test_empty_batch_and_empty_events(h):
    p = h.params(64, 64, 2)
    xy = torch.zeros((0, 2), dtype=torch.int32, device="cuda")
    off = torch.zeros(1, dtype=torch.int64, device="cuda")
    for batched in (False, True):
        out = h.run(xy, off, p, batched=batched)
        assert h.status(out.status) == 0
    ev = gen.generate("plain_small", 5)
    parts = [gen.Events(np.zeros((0, 2), np.int32), np.zeros(1, np.int64), None), ev,
             gen.Events(np.zeros((0, 2), np.int32), np.zeros(2, np.int64), None)]
    cat = gen.concat(parts)
    ref = oracle.run(cat.xy, cat.off, oracle.params(64, 64, 12), threads=THREADS)
    xy, off = dev(cat)
    for batched in (False, True):
        out = h.run(xy, off, h.params(64, 64, 12), checksum=True, batched=batched)
        assert h.status(out.status) == 0
        assert_event_outputs_equal(ref, out.npeaks, out.peaks, out.mask, out.nkept, cat.off, checksum=out.checksum)


def test_bad_hits_and_small_radii(h):
    """r = 0 and out-of-range hits are skipped and flagged; hits inside r ~ 195 mm take the
    int64 path (rho clamped to the edge bins)."""
    rng = np.random.default_rng(9)
    ev = gen.generate("plain_paper", 30)
    xy = ev.xy.copy()
    idx = rng.choice(len(xy), 60, replace=False)
    xy[idx[:10]] = 0
    xy[idx[10:15], 0] = 2 ** 24 + 5
    small = rng.integers(-150000, 150000, size=(45, 2)).astype(np.int32)
    xy[idx[15:]] = small
    ref = oracle.run(xy, ev.off, oracle.params(256, 256, 16, 1, 4096), threads=THREADS)
    assert ref.status == oracle.F_BAD_HIT
    t_xy, off = torch.from_numpy(xy).cuda(), torch.from_numpy(ev.off).cuda()
    for batched in (False, True):
        for tiles in (1, 2):
            out = h.run(t_xy, off, h.params(256, 256, 16, 1, 4096, theta_tiles=tiles), checksum=True, batched=batched)
            assert h.status(out.status) == h.F_BAD_HIT
            assert_event_outputs_equal(ref, out.npeaks, out.peaks, out.mask, out.nkept, ev.off,
                                       checksum=out.checksum)
    st = h.new_status()
    uq, vq = h.map_hits(t_xy, off, st)
    assert h.status(st) == h.F_BAD_HIT
    u = to_np(uq)
    assert np.all(u[idx[:15]] == np.iinfo(np.int64).min)


def test_all_hits_small_radius_event(h):
    """Every hit on the int64 path, across several staging chunks."""
    rng = np.random.default_rng(4)
    xy = rng.integers(-190000, 190000, size=(9000, 2)).astype(np.int32)
    xy[np.all(xy == 0, axis=1)] = 1
    off = np.array([0, 3000, 9000], np.int64)
    ref = oracle.run(xy, off, oracle.params(128, 128, 40, 1, 8192), threads=THREADS)
    t_xy, t_off = torch.from_numpy(xy).cuda(), torch.from_numpy(off).cuda()
    for tiles in (1, 2):
        out = h.run(t_xy, t_off, h.params(128, 128, 40, 1, 8192, theta_tiles=tiles), checksum=True, batched=True)
        assert h.status(out.status) == 0
        assert_event_outputs_equal(ref, out.npeaks, out.peaks, out.mask, out.nkept, off, checksum=out.checksum)


def test_large_event_chunks_and_too_large(h):
    """An event bigger than one staging chunk, and one above 32767 hits (skipped, flagged)."""
    ev = gen.generate("stress", 8)
    big = np.tile(ev.xy, (1, 1))[:32767]
    huge = np.concatenate([ev.xy] * 2)[:32768]
    xy = np.concatenate([big, huge, ev.xy[:500]])
    off = np.array([0, len(big), len(big) + len(huge), len(xy)], np.int64)
    ref = oracle.run(xy, off, oracle.params(256, 256, 200, 1, 4096), threads=THREADS)
    assert ref.status == oracle.F_EVENT_TOO_LARGE
    t_xy, t_off = torch.from_numpy(xy).cuda(), torch.from_numpy(off).cuda()
    for tiles in (1, 4):
        out = h.run(t_xy, t_off, h.params(256, 256, 200, 1, 4096, theta_tiles=tiles), checksum=True, batched=True)
        assert h.status(out.status) == h.F_EVENT_TOO_LARGE
        assert_event_outputs_equal(ref, out.npeaks, out.peaks, out.mask, out.nkept, off, checksum=out.checksum)


def test_bad_offsets_write_nothing(h):
    ev = gen.generate("plain_small", 10)
    bad = ev.off.copy()
    bad[3], bad[4] = bad[4], bad[3]
    xy, off = torch.from_numpy(ev.xy).cuda(), torch.from_numpy(bad).cuda()
    for batched in (False, True):
        out = h.run(xy, off, h.params(64, 64, 12), batched=batched)
        out.npeaks.fill_(-7)
        out.status.zero_()
        h.run(xy, off, h.params(64, 64, 12), out=out, batched=batched)
        assert h.status(out.status) == h.F_BAD_OFFSETS
        assert torch.all(out.npeaks == -7)
    st = h.new_status()
    h.map_hits(xy, off, st)
    assert h.status(st) == h.F_BAD_OFFSETS


def test_peak_overflow_keeps_first_in_raster_order(h):
    cfg = gen.CONFIGS["plain_paper"]
    ev = gen.generate(cfg, 20)
    ref = oracle.run(ev.xy, ev.off, oracle.params(256, 256, 16, 1, 100), threads=THREADS)
    assert ref.status == oracle.F_PEAK_OVERFLOW
    xy, off = dev(ev)
    for tiles in (1, 2, 3, 4):  # 2 and 4: mirror-pair tiles (low and high segments), 3: plain tiles
        out = h.run(xy, off, h.params(256, 256, 16, 1, 100, theta_tiles=tiles), batched=True)
        assert h.status(out.status) == h.F_PEAK_OVERFLOW
        assert_event_outputs_equal(ref, out.npeaks, out.peaks, out.mask, out.nkept, ev.off)


@pytest.mark.parametrize("hw", [0, 3])
def test_keep_halfwidth(h, hw):
    cfg = gen.CONFIGS["plain_paper"]
    ev = gen.generate(cfg, 30)
    ref = oracle.run(ev.xy, ev.off, oracle.params(256, 256, 16, hw, 4096), threads=THREADS)
    xy, off = dev(ev)
    out = h.run(xy, off, h.params(256, 256, 16, hw, 4096), batched=True)
    assert_event_outputs_equal(ref, out.npeaks, out.peaks, out.mask, out.nkept, ev.off)


def test_permutation_invariance_on_gpu(h):
    cfg = gen.CONFIGS["plain_paper"]
    ev = gen.generate(cfg, 20)
    rng = np.random.default_rng(2)
    perm = np.concatenate([ev.off[e] + rng.permutation(ev.off[e + 1] - ev.off[e]) for e in range(20)])
    xy, off = dev(ev)
    a = h.run(xy, off, cfg_params(h, cfg), checksum=True, batched=True)
    b = h.run(torch.from_numpy(ev.xy[perm]).cuda(), off, cfg_params(h, cfg), checksum=True, batched=True)
    assert torch.equal(a.npeaks, b.npeaks) and torch.equal(a.checksum, b.checksum)
    assert np.array_equal(peaks_np(a.peaks), peaks_np(b.peaks))
    assert np.array_equal(to_np(a.mask)[perm], to_np(b.mask))


def test_non_default_stream_and_graph_replay(h):
    cfg = gen.CONFIGS["plain_paper"]
    ev = gen.generate(cfg, 64)
    ref = oracle_of(cfg, ev)
    xy, off = dev(ev)
    s = torch.cuda.Stream()
    out = h.alloc_outputs(ev.n_hits, ev.n_events, cfg_params(h, cfg), checksum=True)
    torch.cuda.synchronize()
    for _ in range(3):  # the second and third calls replay the cached graph
        out.mask.fill_(7)
        with torch.cuda.stream(s):
            h.run(xy, off, cfg_params(h, cfg), out=out, batched=True, stream=s)
        s.synchronize()
        assert_event_outputs_equal(ref, out.npeaks, out.peaks, out.mask, out.nkept, ev.off, checksum=out.checksum)


# ---------------------------------------------------------------- exhaustive bin function

@pytest.mark.parametrize("n_rho", [4, 63, 64, 256, 512, 1000, 1024])
def test_bin_function_exhaustive(h, n_rho):
    """Every rho in [-H - 10^6, H + 10^6]: the device's multiply-high binning equals plain
    64-bit floor division with clamping."""
    H = 703687442
    m = h.selftest_bin(n_rho, -H - 10 ** 6, H + 10 ** 6)
    assert int(m.item()) == 0


@pytest.mark.parametrize("n_theta,n_rho", [(64, 64), (256, 256), (512, 512), (1000, 1000), (1024, 1024), (37, 63)])
def test_float_bin_path_random_tuples(h, n_theta, n_rho):
    """The vote bins through a float estimate and falls back to integer arithmetic when an
    integer lies within the estimate's error bound of it; 2e8 random tuples must all agree
    with exact division, for the general estimate and for the mirror-pair layout's row read
    off the float's bit pattern (whose window is a power of two of 2^-F units, F = 23 - b)."""
    bad, amb, bad_mp, amb_mp, n_mp = h.selftest_fpbin(n_theta, n_rho, 12345 + n_rho, 200_000_000)
    assert bad == 0
    assert 0 < amb < 200_000_000 * 4e-3  # the fallback is exercised, and rare
    assert bad_mp == 0
    assert n_mp > 100_000_000
    b = (n_rho + 1).bit_length()  # 2^b >= n_rho + 2
    assert 0 < amb_mp < n_mp * 2 * 4 * 2.0 ** -(23 - b)  # window of 4 units, twice for slack


def test_autotuned_shape_gives_identical_results(h):
    cfg = gen.CONFIGS["plain_paper"]
    ev = gen.generate(cfg, 200)
    xy, off = dev(ev)
    p = cfg_params(h, cfg)
    tuned, ms = h.autotune(xy, off, p)
    assert ms > 0 and tuned.theta_tiles >= 1 and tuned.block % 32 == 0 and tuned.events_per_cta >= 1
    again, ms2 = h.autotune(xy, off, p)  # cached
    assert ms2 == -1.0 and [getattr(again, f) for f, _ in again._fields_] == [getattr(tuned, f) for f, _ in tuned._fields_]
    ref = oracle_of(cfg, ev)
    out = h.run(xy, off, tuned, checksum=True, batched=True)
    assert h.status(out.status) == 0
    assert_event_outputs_equal(ref, out.npeaks, out.peaks, out.mask, out.nkept, ev.off, checksum=out.checksum)


def test_autotune_cache_keys_the_peak_finder(h):
    """The autotuner writes only the launch shape, and its cache tells the peak finders apart:
    tuning the 3x3 finder first must not hand the iterative finder's tuning the 3x3 parameters.
    (Threshold 17 is used by no other test, so both keys are new to this process.)"""
    cfg = gen.CONFIGS["plain_paper"]
    ev = gen.generate(cfg, 300)
    xy, off = dev(ev)
    algo = ("n_theta", "n_rho", "threshold", "keep_halfwidth", "max_peaks", "peak_mode", "rel_num", "rel_den",
            "nms_radius")
    p0 = h.params(cfg.n_theta, cfg.n_rho, 17, cfg.keep_halfwidth, 512)
    t0, ms0 = h.autotune(xy, off, p0)
    assert ms0 > 0 and [getattr(t0, f) for f in algo] == [getattr(p0, f) for f in algo]
    p1 = h.params(cfg.n_theta, cfg.n_rho, 17, cfg.keep_halfwidth, 512, peak_mode=1, rel_num=1, rel_den=2,
                  nms_radius=3)
    t1, ms1 = h.autotune(xy, off, p1)
    assert ms1 > 0, "the iterative finder's tuning came from the 3x3 finder's cache entry"
    assert [getattr(t1, f) for f in algo] == [getattr(p1, f) for f in algo]
    t1b, ms1b = h.autotune(xy, off, p1)
    assert ms1b == -1.0 and [getattr(t1b, f) for f, _ in t1b._fields_] == [getattr(t1, f) for f, _ in t1._fields_]
    op = oracle.params(cfg.n_theta, cfg.n_rho, 17, cfg.keep_halfwidth, 512, peak_mode=1, rel_num=1, rel_den=2,
                       nms_radius=3)
    ref = oracle.run(ev.xy, ev.off, op, threads=THREADS)
    out = h.run(xy, off, t1, batched=True)
    assert h.status(out.status) == ref.status
    assert_event_outputs_equal(ref, out.npeaks, out.peaks, out.mask, out.nkept, ev.off)


def test_host_errors(h):
    xy = torch.zeros((4, 2), dtype=torch.int32, device="cuda")
    off = torch.tensor([0, 4], dtype=torch.int64, device="cuda")
    for bad in (h.params(3, 64, 2), h.params(64, 1025, 2), h.params(64, 64, 0), h.params(64, 64, 2, max_peaks=0),
                h.params(64, 64, 2, block=48), h.params(64, 64, 2, theta_tiles=65)):
        with pytest.raises(h.HoughError) as ei:
            h.run(xy, off, bad, out=h.alloc_outputs(4, 1, h.params(64, 64, 2)))
        assert ei.value.code == h.EPARAM
    p = h.params(64, 64, 2)
    out = h.alloc_outputs(4, 1, p)
    out.ws = out.ws[:16]
    with pytest.raises(h.HoughError) as ei:
        h.run(xy, off, p, out=out)
    assert ei.value.code == h.EWORKSPACE
    # peak records are written as 8-byte stores: a buffer 2 bytes off is refused before launch
    out = h.alloc_outputs(4, 1, p)
    out.peaks = torch.zeros(4 * p.max_peaks + 4, dtype=torch.int16, device="cuda")[1:]
    for batched in (False, True):
        with pytest.raises(h.HoughError) as ei:
            h.run(xy, off, p, out=out, batched=batched)
        assert ei.value.code == h.EINVAL
    with pytest.raises(h.HoughError) as ei:
        h.run_static(xy, off, p, out)
    assert ei.value.code == h.EINVAL
    # output tensors too small or of the wrong type are refused before anything is enqueued
    out = h.alloc_outputs(4, 1, p)
    out.peaks = out.peaks[:, :10]
    with pytest.raises(ValueError):
        h.run(xy, off, p, out=out)
    out = h.alloc_outputs(4, 1, p)
    out.mask = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(TypeError):
        h.run(xy, off, p, out=out, batched=True)


# ---------------------------------------------------------------- Eq. (2) circle recovery

@pytest.mark.parametrize("name,n", [("plain_paper", 200), ("stress", 20), ("paper_1000", 50)])
def test_circles_match_oracle(h, name, n):
    """Circle of every stored peak (float32 on the GPU from double arithmetic) against the
    oracle's float64, to float rounding; records past each event's stored peaks untouched."""
    cfg = gen.CONFIGS[name]
    ev = gen.generate(cfg, n)
    xy, off = dev(ev)
    p = cfg_params(h, cfg)
    out = h.run(xy, off, p, batched=True)
    circ = torch.full((n, p.max_peaks, 4), -7.0, dtype=torch.float32, device="cuda")
    h.circles(out.npeaks, out.peaks, p, 1.0, out=circ)
    got = to_np(circ)
    npk = np.minimum(to_np(out.npeaks), p.max_peaks)
    pk = to_np(out.peaks)
    for e in range(n):
        recs = pk[e, : npk[e]].astype(np.int16).view(oracle.PEAK_DTYPE).reshape(-1)
        ref = oracle.circles(recs, cfg.n_theta, cfg.n_rho, 1.0)
        np.testing.assert_allclose(got[e, : npk[e]], ref.astype(np.float32), rtol=1e-6, atol=0)
        assert np.all(got[e, npk[e]:] == -7.0)


def test_circles_odd_rho_and_field(h):
    """Odd N_rho has a bin centre at rho = 0 (infinite radius); pT scales with the field."""
    p = h.params(4, 5, 1, 1, 8)
    pk = torch.zeros((1, 8, 4), dtype=torch.int16, device="cuda")
    pk[0, :3, 0] = torch.tensor([0, 1, 3], dtype=torch.int16)
    pk[0, :3, 1] = torch.tensor([0, 2, 4], dtype=torch.int16)
    npk = torch.tensor([3], dtype=torch.int32, device="cuda")
    got = to_np(h.circles(npk, pk, p, 1.5))[0, :3]
    recs = to_np(pk)[0, :3].view(oracle.PEAK_DTYPE).reshape(-1)
    ref = oracle.circles(recs, 4, 5, 1.5).astype(np.float32)
    assert np.isinf(got[1, 2]) and np.isinf(got[1, 3]) and np.isinf(ref[1, 2])
    fin = np.isfinite(ref)
    np.testing.assert_allclose(got[fin], ref[fin], rtol=1e-6)
    assert np.array_equal(np.sign(got[~fin]), np.sign(ref[~fin]))


# ---------------------------------------------------------------- iterative peak finder (Sec. 2)

ITER = [  # (workload, events, n_theta, n_rho, threshold, rel_num, rel_den, nms_radius, max_peaks)
    ("plain_paper", 60, 256, 256, 16, 1, 2, 3, 64),
    ("plain_paper", 40, 64, 64, 8, 1, 3, 1, 256),
    ("batched", 60, 256, 256, 16, 2, 5, 2, 128),
    ("plain_small", 30, 64, 64, 6, 0, 1, 0, 300),    # no relative cut, no neighbourhood: every cell >= T
    ("plain_paper", 30, 100, 63, 8, 1, 4, 2, 512),   # N_theta not a multiple of 64, odd N_rho
    ("plain_paper", 20, 256, 256, 16, 1, 10, 1, 8),  # overflow: more peaks than stored
    # 20k-40k candidates an event, above the sorted form's 8,192 keys: one pass per peak
    ("batched", 12, 256, 256, 4, 0, 1, 6, 512),
    # 1k-10k candidates: events of both forms in one launch, sorts of up to 8,192 keys
    ("batched", 40, 256, 256, 16, 1, 3, 3, 1024),
]


@pytest.mark.parametrize("name,n,nt,nr,thr,num,den,R,mx", ITER)
def test_iterative_fused_and_stepwise_match_oracle(h, name, n, nt, nr, thr, num, den, R, mx):
    cfg = gen.CONFIGS[name]
    ev = gen.generate(cfg, n)
    op = oracle.params(nt, nr, thr, 1, mx, peak_mode=1, rel_num=num, rel_den=den, nms_radius=R)
    ref = oracle.run(ev.xy, ev.off, op, with_acc=True, threads=THREADS)
    xy, off = dev(ev)
    p = h.params(nt, nr, thr, 1, mx, peak_mode=1, rel_num=num, rel_den=den, nms_radius=R)
    for batched in (False, True):
        out = h.run(xy, off, p, checksum=True, batched=batched)
        assert h.status(out.status) == ref.status
        assert_event_outputs_equal(ref, out.npeaks, out.peaks, out.mask, out.nkept, ev.off, checksum=out.checksum)
    # stepwise: the iterative finder on the oracle's accumulator in HBM
    st = h.new_status()
    acc = torch.from_numpy(ref.acc).cuda()
    npk, pk = h.peaks(acc, p, st)
    assert np.array_equal(to_np(npk), ref.npeaks)
    assert np.array_equal(peaks_np(pk), peaks_np(torch.from_numpy(ref.peaks.view(np.int16).reshape(n, mx, 4))))


def test_iterative_cell_above_4095_votes(h):
    """4,200 copies of one hit put 4,200 votes into a cell of every column: beyond the 12-bit vote
    field of the sorted form's keys, so that event takes one pass per peak; its neighbours in the
    batch take the sorted form. Fused, batched and stepwise results as the oracle's."""
    ev = gen.generate(gen.CONFIGS["plain_paper"], 3)
    a, b = int(ev.off[1]), int(ev.off[2])
    xy = np.concatenate([ev.xy[:b], np.repeat(ev.xy[a:a + 1], 4200, axis=0), ev.xy[b:]])
    off = ev.off.copy()
    off[2:] += 4200
    n_t, n_r = 128, 128
    op = oracle.params(n_t, n_r, 10, 1, 512, peak_mode=1, rel_num=1, rel_den=2, nms_radius=2)
    ref = oracle.run(xy, off, op, with_acc=True, threads=THREADS)
    assert ref.acc.reshape(3, n_t, n_r)[1].max() >= 4200
    p = h.params(n_t, n_r, 10, 1, 512, peak_mode=1, rel_num=1, rel_den=2, nms_radius=2)
    d_xy, d_off = torch.from_numpy(xy).cuda(), torch.from_numpy(off).cuda()
    for batched in (False, True):
        out = h.run(d_xy, d_off, p, checksum=True, batched=batched)
        assert h.status(out.status) == ref.status
        assert_event_outputs_equal(ref, out.npeaks, out.peaks, out.mask, out.nkept, off, checksum=out.checksum)
    npk, pk = h.peaks(torch.from_numpy(ref.acc).cuda(), p, h.new_status())
    assert np.array_equal(to_np(npk), ref.npeaks)
    assert np.array_equal(peaks_np(pk), peaks_np(torch.from_numpy(ref.peaks.view(np.int16).reshape(3, 512, 4))))


def test_iterative_stepwise_large_accumulator(h):
    """1000 x 1000 (2 MB accumulator, no single-CTA fused plan): the stepwise finder keeps its
    suppression bitmap in shared memory."""
    cfg = gen.CONFIGS["paper_1000"]
    ev = gen.generate(cfg, 6)
    op = oracle.params(1000, 1000, 12, 1, 256, peak_mode=1, rel_num=1, rel_den=2, nms_radius=4)
    ref = oracle.run(ev.xy, ev.off, op, with_acc=True, threads=THREADS)
    p = h.params(1000, 1000, 12, 1, 256, peak_mode=1, rel_num=1, rel_den=2, nms_radius=4)
    st = h.new_status()
    npk, pk = h.peaks(torch.from_numpy(ref.acc).cuda(), p, st)
    assert h.status(st) == 0
    assert np.array_equal(to_np(npk), ref.npeaks)
    n = ref.npeaks
    got = peaks_np(pk)
    exp = peaks_np(torch.from_numpy(ref.peaks.view(np.int16).reshape(len(n), 256, 4)))
    for e in range(len(n)):
        assert np.array_equal(got[e][: min(n[e], 256)], exp[e][: min(n[e], 256)])


# ---------------------------------------------------------------- iterative finder on theta tiles

ITER_TILED = [  # (workload, events, n_theta, n_rho, threshold, rel_num, rel_den, nms_radius, max_peaks, tiles)
    ("plain_paper", 40, 256, 256, 16, 1, 2, 3, 2048, 2),
    ("plain_paper", 30, 256, 256, 16, 1, 2, 3, 2048, 4),   # windows across three tile edges
    ("stress", 8, 512, 512, 20, 1, 2, 3, 16384, 4),        # the stress shape (13k candidates an event)
    ("plain_paper", 20, 101, 63, 8, 1, 4, 2, 512, 3),      # odd N_theta: column tiles, no mirror pairs
    ("plain_paper", 12, 1000, 1000, 12, 1, 2, 4, 1024, 16),  # the paper's discretisation
    ("plain_small", 20, 64, 64, 6, 0, 1, 0, 300, 2),       # every cell >= T, no neighbourhood
    ("batched", 16, 256, 256, 16, 1, 2, 64, 256, 8),       # windows wider than a tile (R = 64)
]


def run_iterative_tiled(h, xy_np, off_np, nt, nr, thr, num, den, R, mx, tiles):
    op = oracle.params(nt, nr, thr, 1, mx, peak_mode=1, rel_num=num, rel_den=den, nms_radius=R)
    ref = oracle.run(xy_np, off_np, op, threads=THREADS)
    xy, off = torch.from_numpy(xy_np).cuda(), torch.from_numpy(off_np).cuda()
    p = h.params(nt, nr, thr, 1, mx, theta_tiles=tiles, peak_mode=1, rel_num=num, rel_den=den, nms_radius=R)
    assert h.resolve(p).theta_tiles == tiles
    deferred = []
    for batched in (False, True):
        out = h.run(xy, off, p, checksum=True, batched=batched)
        assert h.status(out.status) == ref.status
        assert_event_outputs_equal(ref, out.npeaks, out.peaks, out.mask, out.nkept, off_np, checksum=out.checksum)
        deferred.append(int(out.ws[8:12].view(torch.int32).item()))  # events the fallback kernel took
    return ref, deferred


@pytest.mark.parametrize("name,n,nt,nr,thr,num,den,R,mx,tiles", ITER_TILED)
def test_iterative_tiled_matches_oracle(h, name, n, nt, nr, thr, num, den, R, mx, tiles):
    """The paper's iterative finder with the accumulator split over theta tiles: each tile
    publishes its candidates, the last tile of the event settles them; fused and batched
    launches, outputs and accumulator checksums equal the oracle's."""
    ev = gen.generate(gen.CONFIGS[name], n)
    run_iterative_tiled(h, ev.xy, ev.off, nt, nr, thr, num, den, R, mx, tiles)


def test_iterative_tiled_deferred_events(h):
    """Events whose candidates do not fit the tiles' record slots (max_peaks 32 here) go to the
    fallback kernel (HBM accumulator, the stepwise finder): results still equal the oracle's,
    peak-list overflow included, and the fallback really ran."""
    ev = gen.generate(gen.CONFIGS["plain_paper"], 24)
    ref, deferred = run_iterative_tiled(h, ev.xy, ev.off, 256, 256, 16, 1, 2, 3, 32, 4)
    assert min(deferred) > 0 and ref.status & 4  # some events deferred; some peak lists overflowed


def test_iterative_tiled_cell_above_4095_votes(h):
    """A cell above 4,095 votes (beyond the candidate keys' vote field) defers its event; its
    neighbours in the batch take the tiles' candidate lists."""
    ev = gen.generate(gen.CONFIGS["plain_paper"], 3)
    a, b = int(ev.off[1]), int(ev.off[2])
    xy = np.concatenate([ev.xy[:b], np.repeat(ev.xy[a:a + 1], 4200, axis=0), ev.xy[b:]])
    off = ev.off.copy()
    off[2:] += 4200
    _, deferred = run_iterative_tiled(h, xy, off, 256, 256, 10, 1, 2, 2, 4096, 2)
    assert deferred == [1, 1]  # the event with the 4,200-vote cells, in both launches


@pytest.mark.parametrize("name,sample", [("stress", 40), ("paper_1000", 80)])
def test_full_size_sampled_iterative_tiled(h, name, sample):
    """The stress (512 x 512) and 1000 x 1000 workloads, whole, with the iterative finder (half the
    maximum, radius 3) in the autotuned launch shape; the oracle recomputes a random sample."""
    cfg = gen.CONFIGS[name]
    ev = gen.generate(cfg, with_truth=False)
    xy, off = dev(ev)
    kw = dict(peak_mode=1, rel_num=1, rel_den=2, nms_radius=3)
    p = cfg_params(h, cfg, **kw)
    ns = min(ev.n_events, 2000)
    p, _ = h.autotune(xy[: int(ev.off[ns])], off[: ns + 1], p)
    assert h.resolve(p).theta_tiles > 1
    out = h.run(xy, off, p, checksum=False, batched=True)
    assert h.status(out.status) == 0
    rng = np.random.default_rng(3)
    events = np.sort(rng.choice(ev.n_events, size=sample, replace=False))
    events[0] = 0
    events[-1] = ev.n_events - 1
    sxy, soff = sub_batch(ev.xy, ev.off, events)
    ref = oracle.run(sxy, soff, oracle.params(cfg.n_theta, cfg.n_rho, cfg.threshold, cfg.keep_halfwidth,
                                              cfg.max_peaks, **kw), threads=THREADS)
    assert_event_outputs_equal(ref, out.npeaks, out.peaks, out.mask, out.nkept, ev.off, events=events)


# ---------------------------------------------------------------- host-buffer path (pipelined chunks)

@pytest.mark.parametrize("name,n,iterative", [("plain_paper", 300, False), ("batched", 9000, False),
                                               ("stress", 4100, False), ("batched", 5000, True)])
def test_host_path_matches_oracle(h, name, n, iterative):
    """hough_run_host: pinned host inputs in, host results out. 9,000, 5,000 and 4,100 events run
    as several pipelined chunks (rebased offsets, peaks packed per chunk and re-based on the
    host); also with the iterative finder (half the maximum, radius 3)."""
    cfg = gen.CONFIGS[name]
    ev = gen.generate(cfg, n)
    kw = dict(peak_mode=1, rel_num=1, rel_den=2, nms_radius=3) if iterative else {}
    ref = oracle.run(ev.xy, ev.off, oracle.params(cfg.n_theta, cfg.n_rho, cfg.threshold, cfg.keep_halfwidth,
                                                  cfg.max_peaks, **kw), threads=THREADS)
    p = cfg_params(h, cfg, **kw)
    r = h.HostRunner(ev.n_hits, ev.n_events, p)
    xy = torch.from_numpy(ev.xy).pin_memory()
    off = torch.from_numpy(ev.off).pin_memory()
    for _ in range(2):  # a second call reuses the cached graphs and streams
        assert r(xy, off) == 0
        assert np.array_equal(r.npeaks.numpy(), ref.npeaks)
        assert np.array_equal(r.nkept.numpy(), ref.nkept)
        assert np.array_equal(r.mask.numpy()[: ev.n_hits], ref.mask)
        po = r.peak_off.numpy()
        stored = np.minimum(ref.npeaks, cfg.max_peaks)
        assert po[0] == 0 and np.array_equal(np.diff(po), stored)
        dense = r.peaks.numpy()[: po[-1]].astype(np.int16).view(oracle.PEAK_DTYPE).reshape(-1)
        for e in range(n):
            assert np.array_equal(dense[po[e]: po[e + 1]], ref.peaks[e, : stored[e]]), e


def test_host_path_errors(h):
    cfg = gen.CONFIGS["plain_paper"]
    ev = gen.generate(cfg, 50)
    p = cfg_params(h, cfg)
    xy = torch.from_numpy(ev.xy).pin_memory()
    off = torch.from_numpy(ev.off).pin_memory()
    small = h.HostRunner(ev.n_hits, ev.n_events, p, peaks_cap=10)
    with pytest.raises(h.HoughError) as ei:
        small(xy, off)
    assert ei.value.code == h.EWORKSPACE
    ref = oracle_of(cfg, ev)
    assert np.array_equal(small.npeaks.numpy(), ref.npeaks)  # counts and offsets still valid
    assert small.peak_off.numpy()[-1] == np.minimum(ref.npeaks, cfg.max_peaks).sum()
    bad = off.clone()
    bad[10] = bad[11] + 1  # offsets must not decrease: refused on the host, nothing enqueued
    r = h.HostRunner(ev.n_hits, ev.n_events, p)
    with pytest.raises(h.HoughError) as ei:
        r(xy, bad)
    assert ei.value.code == h.EINVAL
