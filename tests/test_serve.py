"""Serving loop (continuous batching), checked against the CPU oracle: every served event's
peaks, counts and kept mask equal the oracle's for both peak finders, alone and inside a mix of
other events; a replayed Poisson stream copies every request's results out and each equals the
oracle's result for its event; admission refuses beyond the queue capacity; a micro-batch whose
launch fails reports no result as OK; the loop's batch records are consistent."""
import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ITERATIVE = dict(peak_mode=1, rel_num=1, rel_den=2, nms_radius=3)


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_04067_gb300 as hough
    hough.load()
    return hough


def cfg_params(h, cfg, iterative=False, max_peaks=None):
    kw = ITERATIVE if iterative else {}
    return h.params(cfg.n_theta, cfg.n_rho, cfg.threshold, cfg.keep_halfwidth, max_peaks or cfg.max_peaks, **kw)


def oracle_ref(cfg, ev, iterative=False, max_peaks=None):
    kw = ITERATIVE if iterative else {}
    p = oracle.params(cfg.n_theta, cfg.n_rho, cfg.threshold, cfg.keep_halfwidth, max_peaks or cfg.max_peaks, **kw)
    return oracle.run(ev.xy, ev.off, p, threads=8)


def assert_matches_oracle(ref, ev, e, npeaks, nkept, mask, pk, maxp):
    """Served event e's outputs against the oracle's event e, element by element."""
    assert npeaks == ref.npeaks[e], (e, npeaks, ref.npeaks[e])
    assert nkept == ref.nkept[e], (e, nkept, ref.nkept[e])
    assert np.array_equal(mask, ref.mask[ev.off[e]:ev.off[e + 1]]), e
    s = min(int(ref.npeaks[e]), maxp)
    got = np.ascontiguousarray(pk[:s]).view(oracle.PEAK_DTYPE).reshape(-1)
    assert np.array_equal(got, ref.peaks[e, :s]), e


def serve_events(srv, ev, ids, maxp):
    """Submits events (by index) and returns {event: (npeaks, nkept, mask, peaks, status)}."""
    out = {}
    bufs = []
    for rid, e in enumerate(ids):
        xy = np.ascontiguousarray(ev.xy[ev.off[e]:ev.off[e + 1]])
        mask = np.full(len(xy), 7, np.uint8)  # sentinel: a result must overwrite it
        pk = np.zeros((maxp, 4), np.int16)
        bufs.append((xy, mask, pk))
        assert srv.submit(xy, rid, mask, pk) == 0
    srv.drain(60)
    res = srv.poll()
    assert len(res) == len(ids)
    for r in res:
        xy, mask, pk = bufs[r.id]
        out[ids[r.id]] = (r.npeaks, r.nkept, mask.copy(), pk.copy(), r.status)
    return out


@pytest.mark.parametrize("iterative", [False, True])
def test_served_events_match_oracle(h, iterative):
    cfg = gen.CONFIGS["served"]
    ev = gen.generate(cfg, 300)
    p = cfg_params(h, cfg, iterative)
    ref = oracle_ref(cfg, ev, iterative)
    with h.Server(p, slots=3, max_batch_events=40, flush_us=100) as srv:
        got = serve_events(srv, ev, list(range(ev.n_events)), cfg.max_peaks)
    for e in range(ev.n_events):
        g_np, g_nk, g_mask, g_pk, st = got[e]
        assert st == 0
        assert_matches_oracle(ref, ev, e, g_np, g_nk, g_mask, g_pk, cfg.max_peaks)


@pytest.mark.parametrize("iterative", [False, True])
def test_alone_equals_in_the_mix_equals_oracle(h, iterative):
    cfg = gen.CONFIGS["served"]
    ev = gen.generate(cfg, 120)
    p = cfg_params(h, cfg, iterative)
    ref = oracle_ref(cfg, ev, iterative)
    probe = [3, 57, 101]
    with h.Server(p, slots=4, max_batch_events=32, flush_us=50) as srv:
        alone = {e: serve_events(srv, ev, [e], cfg.max_peaks)[e] for e in probe}
        rng = np.random.default_rng(0)
        mix_ids = list(rng.permutation(ev.n_events))
        mixed = serve_events(srv, ev, mix_ids, cfg.max_peaks)
    for e in range(ev.n_events):
        assert mixed[e][4] == 0
        assert_matches_oracle(ref, ev, e, *mixed[e][:4], cfg.max_peaks)
    for e in probe:
        a, m = alone[e], mixed[e]
        assert a[4] == 0
        assert_matches_oracle(ref, ev, e, *a[:4], cfg.max_peaks)
        assert a[0] == m[0] and a[1] == m[1] and np.array_equal(a[2], m[2])


def test_admission_refuses_when_queue_full(h):
    cfg = gen.CONFIGS["served"]
    ev = gen.generate(cfg, 8)
    p = cfg_params(h, cfg)
    # flush only when full (never, with these sizes) and room for 4 waiting requests
    with h.Server(p, slots=1, max_batch_events=64, flush_us=0, queue_capacity=4) as srv:
        xys = [np.ascontiguousarray(ev.xy[ev.off[e]:ev.off[e + 1]]) for e in range(8)]
        rcs = [srv.submit(xys[e], e) for e in range(8)]
        assert rcs[:4] == [0, 0, 0, 0] and all(rc == h.EFULL for rc in rcs[4:])
        srv.drain(30)  # drain launches the partial batch
        assert sorted(r.id for r in srv.poll()) == [0, 1, 2, 3]


def test_replayed_poisson_stream_matches_oracle(h):
    """Requests arrive as a Poisson stream (100 k events/s) from a pool of events; every request's
    mask and peaks are copied out by the loop and compared with the oracle's for its event."""
    cfg = gen.CONFIGS["served"]
    pool = gen.generate(cfg, 1000, with_truth=False)
    maxp = cfg.max_peaks  # above every pool event's peak count (checked below)
    p = cfg_params(h, cfg, max_peaks=maxp)
    ref = oracle_ref(cfg, pool, max_peaks=maxp)
    assert ref.npeaks.max() <= maxp
    rate, n = 100_000, 3000
    rng = np.random.default_rng(7)
    arrival = np.cumsum(rng.exponential(1e9 / rate, size=n)).astype(np.int64)
    ev_of = np.arange(n) % pool.n_events
    sizes = np.diff(pool.off)[ev_of]
    moff = np.zeros(n + 1, np.int64)
    moff[1:] = np.cumsum(sizes)
    mask = np.full(int(moff[-1]), 7, np.uint8)
    peaks = np.zeros((n, maxp, 4), np.int16)
    with h.Server(p, slots=4, max_batch_events=128, flush_us=50) as srv:
        srv.replay(pool.xy, pool.off, arrival, mask_out=mask, peaks_out=peaks)
        srv.drain(60)
        res = srv.poll_numpy(n + 16)
        stats, rec = srv.trace()
    assert len(res) == n and np.all(res["status"] == 0)
    lat = (res["t_done_ns"] - res["t_arrival_ns"]) / 1e3
    assert np.all(lat > 0) and np.percentile(lat, 99) < 50_000  # microseconds
    by_id = np.argsort(res["id"])
    res = res[by_id]
    assert np.array_equal(res["id"], np.arange(n))
    for i in range(n):
        e = int(ev_of[i])
        assert_matches_oracle(ref, pool, e, int(res["npeaks"][i]), int(res["nkept"][i]), mask[moff[i]:moff[i + 1]],
                              peaks[i], maxp)
    # the loop's batch records account for every request, in order of launch
    assert stats["batches"] == len(rec) and int(rec["n_events"].sum()) == n
    assert np.all(rec["t_gather"] <= rec["t_launched"]) and np.all(rec["t_launched"] <= rec["t_done_seen"])
    assert np.all(rec["t_done_seen"] <= rec["t_finished"]) and np.all(np.diff(rec["t_gather"]) >= 0)
    assert int(rec["n_hits"].sum()) == int(sizes.sum())
    assert stats["passes"] > 0 and stats["stall_ns"] == 1_000_000


def test_replay_results_into_caller_array(h):
    """With a result array, the replay's requests deliver their records there (by request id),
    nothing reaches poll(), and the counts equal the oracle's for every request."""
    cfg = gen.CONFIGS["served"]
    pool = gen.generate(cfg, 500, with_truth=False)
    p = cfg_params(h, cfg)
    ref = oracle_ref(cfg, pool)
    n = 2500
    arrival = np.cumsum(np.random.default_rng(3).exponential(1e9 / 200_000, size=n)).astype(np.int64)
    res = h.Server.result_array(n)
    with h.Server(p, slots=4, max_batch_events=64, flush_us=50, queue_capacity=256) as srv:
        srv.replay(pool.xy, pool.off, arrival, results_out=res)
        srv.drain(60)
        assert len(srv.poll()) == 0
    ev_of = np.arange(n) % pool.n_events
    assert np.array_equal(res["id"], np.arange(n)) and np.all(res["status"] == 0)
    assert np.array_equal(res["npeaks"], ref.npeaks[ev_of]) and np.array_equal(res["nkept"], ref.nkept[ev_of])
    assert np.all(res["t_done_ns"] > res["t_arrival_ns"])


def test_failed_launch_reports_no_result_as_ok(h):
    """A micro-batch whose launch fails (a host-side injected CUDA error, before anything is
    enqueued) finishes its requests with F_LAUNCH_FAILED, zero counts and untouched output
    buffers; the server keeps serving, and the later requests equal the oracle."""
    cfg = gen.CONFIGS["served"]
    ev = gen.generate(cfg, 40)
    p = cfg_params(h, cfg)
    ref = oracle_ref(cfg, ev)
    with h.Server(p, slots=2, max_batch_events=10, flush_us=0) as srv:
        srv.inject_launch_failures(1)
        first = serve_events(srv, ev, list(range(10)), cfg.max_peaks)  # one full batch: the failed one
        rest = serve_events(srv, ev, list(range(10, 40)), cfg.max_peaks)
    for e, (npk, nk, mask, pk, st) in first.items():
        assert st == h.F_LAUNCH_FAILED and npk == 0 and nk == 0
        assert np.all(mask == 7) and not pk.any()  # nothing was written
    for e, (npk, nk, mask, pk, st) in rest.items():
        assert st == 0
        assert_matches_oracle(ref, ev, e, npk, nk, mask, pk, cfg.max_peaks)
