"""Host-side checks of the C ABI library (no GPU needed): it loads, exports every entry
point include/hough.h declares, validates parameters and plans launch shapes."""
import ctypes
import re

import pytest

import paper_2607_04067_gb300 as h


@pytest.fixture(scope="module")
def lib():
    return h.load()


def test_exports_every_declared_symbol(lib):
    syms = h.declared_symbols()
    assert len(syms) >= 13
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing
    with open(h.HEADER) as f:
        text = f.read()
    # every declaration is inside extern "C" and uses no C++ types
    assert 'extern "C"' in text
    code = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    assert not re.search(r"\b(torch|at::|std::|cudaStream_t|cudaEvent_t)\b", code)


def test_strerror_and_codes(lib):
    for code in (0, -1, -2, -3, -4, -5, -6, -7, -8, 1, 2, 4, 8, 16):
        s = lib.hough_strerror(code)
        assert s and b"unknown" not in s
    assert b"unknown" in lib.hough_strerror(12345)


def test_resolve_and_reject_params():
    r = h.resolve(h.params(256, 256, 16, max_peaks=4096))
    assert r.theta_tiles == 1 and r.block % 32 == 0
    r = h.resolve(h.params(512, 512, 20, max_peaks=16384))
    assert r.theta_tiles >= 2  # 512 x 512 int16 = 512 KB does not fit one CTA
    r = h.resolve(h.params(1024, 1024, 20))
    assert r.theta_tiles >= 5
    r = h.resolve(h.params(256, 256, 16, theta_tiles=4, block=0))
    assert r.theta_tiles == 4 and r.block == 2 * 32 * (r.block // 64) + 32 or r.block <= 1024
    for bad in (h.params(3, 64, 1), h.params(64, 2000, 1), h.params(64, 64, 0), h.params(64, 64, 1, -1),
                h.params(64, 64, 1, max_peaks=0), h.params(64, 64, 1, theta_tiles=100), h.params(64, 64, 1, block=33),
                h.params(64, 64, 1, peak_mode=2), h.params(64, 64, 1, peak_mode=1, rel_den=0),
                h.params(64, 64, 1, peak_mode=1, rel_num=3, rel_den=2),
                h.params(64, 64, 1, peak_mode=1, nms_radius=32), h.params(64, 64, 1, peak_mode=1, nms_radius=-1)):
        with pytest.raises(h.HoughError) as ei:
            h.resolve(bad)
        assert ei.value.code == h.EPARAM
    # the iterative finder: the whole accumulator in one CTA where it fits, else theta tiles
    r = h.resolve(h.params(256, 256, 16, max_peaks=4096, peak_mode=1, rel_num=1, rel_den=2, nms_radius=3))
    assert r.theta_tiles == 1 and r.peak_mode == 1 and r.rel_den == 2 and r.nms_radius == 3
    assert h.resolve(h.params(256, 256, 16, peak_mode=1, theta_tiles=2)).theta_tiles == 2
    assert h.resolve(h.params(512, 512, 20, peak_mode=1, rel_num=1, rel_den=2)).theta_tiles == 4


def test_workspace_sizes(lib):
    small = h.workspace_size(h.params(256, 256, 16, max_peaks=4096), 1000)
    big = h.workspace_size(h.params(256, 256, 16, max_peaks=4096), 100000)
    assert 0 < small < big
    tiled = h.workspace_size(h.params(256, 256, 16, max_peaks=100, theta_tiles=4), 1000)
    assert tiled >= 1000 * 4 * 100 * 8  # per-tile peak slots
    p = h.params(64, 64, 12)
    assert lib.hough_host_buffer_size(ctypes.byref(p), 1000, 10) >= 1000 * 9


def test_bin_magic_exact_at_every_bin_edge():
    """The device bins t = rho + H with floor(t * M / 2^64), M = ceil(2^64 N / 2H). The only
    places it could differ from floor(t N / 2H) are just below a bin edge; check every edge
    for a range of N with exact integers (the GPU test sweeps every t)."""
    H = 703687442
    two_h = 2 * H
    assert two_h * two_h < 2 ** 64
    for n in (4, 7, 63, 64, 100, 255, 256, 257, 500, 512, 999, 1000, 1023, 1024):
        M = -(-(2 ** 64 * n) // two_h)
        assert M < 2 ** 44
        for k in range(1, n + 1):
            edge = -(-(k * two_h) // n)  # smallest t with floor(t N / 2H) >= k
            for t in (edge - 2, edge - 1, edge, edge + 1):
                if 0 <= t < two_h:
                    assert (t * M) >> 64 == (t * n) // two_h


def test_phase_counters_off_in_the_default_build(lib):
    """hough_phase_cycles needs no GPU in the default build: it reports the timers as off and
    writes zeros; bad arguments are refused."""
    enabled, cyc = h.phase_cycles(reset=True)
    assert enabled is False and set(cyc) == set(h.PHASES) and not any(cyc.values())
    assert lib.hough_phase_cycles(None, 4, 0, None) == -1
    buf = (ctypes.c_uint64 * 4)()
    assert lib.hough_phase_cycles(buf, -1, 0, None) == -1
    # the header's phase numbering is the binding's
    with open(h.HEADER) as f:
        text = f.read()
    ids = dict((m.group(1).lower(), int(m.group(2))) for m in re.finditer(r"#define HOUGH_PHASE_(\w+) (\d+)", text))
    assert ids.pop("count") == len(h.PHASES)
    assert [name for name, _ in sorted(ids.items(), key=lambda kv: kv[1])] == list(h.PHASES)


# theta tiles the plan takes for each accumulator shape (n_theta, n_rho), for both peak finders;
# shapes not listed fit one CTA (one tile)
PLAN_TILES = {(100, 1000): 2, (100, 1024): 2, (256, 1000): 4, (256, 1024): 4, (300, 1000): 5, (300, 1024): 5,
              (512, 256): 2, (512, 1000): 8, (512, 1024): 8, (1000, 256): 4, (1000, 1000): 16, (1000, 1024): 16,
              (1024, 256): 4, (1024, 1000): 16, (1024, 1024): 16}


@pytest.mark.parametrize("nt", [4, 8, 64, 100, 256, 300, 512, 1000, 1024])
@pytest.mark.parametrize("nr", [4, 63, 256, 1000, 1024])
def test_plans_over_shapes(nt, nr):
    """Every accumulator shape has a plan for both peak finders, theta-tiled exactly where one CTA
    cannot hold the accumulator (the iterative finder merges its tiles' candidates)."""
    expect = PLAN_TILES.get((nt, nr), 1)
    for kw in ({}, dict(peak_mode=h.PEAK_ITERATIVE, rel_num=1, rel_den=2, nms_radius=1)):
        r = h.resolve(h.params(nt, nr, 16, 1, 1024, **kw))
        assert r.theta_tiles == expect, (kw, r.theta_tiles)
        assert r.block % 32 == 0 and 32 <= r.block <= 1024 and r.events_per_cta >= 1


def test_probe_rejects_bad_arguments(lib):
    """The shared-atomic probe checks its arguments before anything is launched (no GPU needed):
    modes 0-4 exist, and the array must fit the shared-memory budget."""
    sink = ctypes.c_void_p(256)  # never dereferenced: every call below is refused first
    for mode, ctas, threads, smem, iters in ((5, 2, 1024, 98304, 10), (-1, 2, 1024, 98304, 10),
                                            (0, 0, 1024, 98304, 10), (0, 2, 1000, 98304, 10),
                                            (0, 2, 1024, 1024, 10), (0, 2, 1024, 1 << 20, 10), (4, 2, 1024, 98304, 0)):
        assert lib.hough_probe_smem_atomics(mode, ctas, threads, smem, iters, sink, None) == h.EINVAL
    assert lib.hough_probe_smem_atomics(0, 2, 1024, 98304, 10, None, None) == h.EINVAL
