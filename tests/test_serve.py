"""Serving loop (continuous batching): results equal the batched path's, each event's result is
the same alone and inside a mix of other events, admission refuses beyond the queue capacity,
and a replayed Poisson stream completes with finite latencies."""
import numpy as np
import pytest

import gen
from parity_util import peaks_np, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_04067_gb300 as hough
    hough.load()
    return hough


def cfg_params(h, cfg):
    return h.params(cfg.n_theta, cfg.n_rho, cfg.threshold, cfg.keep_halfwidth, cfg.max_peaks)


def serve_events(h, srv, ev, ids, maxp):
    """Submits events (by index) and returns {event: (npeaks, nkept, mask, peaks, status)}."""
    out = {}
    bufs = []
    for rid, e in enumerate(ids):
        xy = np.ascontiguousarray(ev.xy[ev.off[e]:ev.off[e + 1]])
        mask = np.zeros(len(xy), np.uint8)
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
def test_serve_matches_batched_path(h, iterative):
    cfg = gen.CONFIGS["served"]
    ev = gen.generate(cfg, 300)
    p = cfg_params(h, cfg)
    if iterative:  # the paper's iterative peak finder through the serving loop
        p.peak_mode, p.rel_num, p.rel_den, p.nms_radius = h.PEAK_ITERATIVE, 1, 2, 3
    ref = h.run(torch.from_numpy(ev.xy).cuda(), torch.from_numpy(ev.off).cuda(), p, batched=True)
    npk, nk, mk, pk = to_np(ref.npeaks), to_np(ref.nkept), to_np(ref.mask), peaks_np(ref.peaks)
    with h.Server(p, slots=3, max_batch_events=40, flush_us=100) as srv:
        got = serve_events(h, srv, ev, list(range(ev.n_events)), cfg.max_peaks)
    for e in range(ev.n_events):
        g_np, g_nk, g_mask, g_pk, st = got[e]
        assert st == 0
        assert g_np == npk[e] and g_nk == nk[e]
        assert np.array_equal(g_mask, mk[ev.off[e]:ev.off[e + 1]])
        s = min(g_np, cfg.max_peaks)
        assert np.array_equal(g_pk[:s].view(pk.dtype).reshape(-1), pk[e, :s]), e


def test_alone_equals_in_the_mix(h):
    cfg = gen.CONFIGS["served"]
    ev = gen.generate(cfg, 120)
    p = cfg_params(h, cfg)
    probe = [3, 57, 101]
    with h.Server(p, slots=4, max_batch_events=32, flush_us=50) as srv:
        alone = {e: serve_events(h, srv, ev, [e], cfg.max_peaks)[e] for e in probe}
        rng = np.random.default_rng(0)
        mix_ids = list(rng.permutation(ev.n_events))
        mixed = serve_events(h, srv, ev, mix_ids, cfg.max_peaks)
    for e in probe:
        a, m = alone[e], mixed[e]
        assert a[0] == m[0] and a[1] == m[1]
        assert np.array_equal(a[2], m[2]) and np.array_equal(a[3][:min(a[0], cfg.max_peaks)],
                                                             m[3][:min(m[0], cfg.max_peaks)])


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


def test_replayed_poisson_stream(h):
    cfg = gen.CONFIGS["served"]
    pool = gen.generate(cfg, 2000, with_truth=False)
    p = cfg_params(h, cfg)
    rate, seconds = 100_000, 0.3
    rng = np.random.default_rng(7)
    gaps = rng.exponential(1e9 / rate, size=int(rate * seconds))
    arrival = np.cumsum(gaps).astype(np.int64)
    with h.Server(p, slots=4, max_batch_events=128, flush_us=200) as srv:
        srv.replay(pool.xy, pool.off, arrival)
        srv.drain(60)
        res = srv.poll_numpy()
    assert len(res) == len(arrival)
    lat = (res["t_done_ns"] - res["t_arrival_ns"]) / 1e3
    assert np.all(lat > 0) and np.percentile(lat, 99) < 50_000  # microseconds
    assert np.all(res["status"] == 0)
