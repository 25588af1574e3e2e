"""Pins of the CPU oracle against what the paper and mathematics fix (no GPU).

P1 closed form (Eq. 1-2 and the Hough line relation of Sec. 2), P2 vote/peak/select
invariants, P3 brute force against an independent big-integer restatement, P5
hand-built peak cases, P6 hit-permutation invariance, and the constants of the
paper's discretisation (Sec. 2) and of the checksum's published hash.
"""
import math
import os
import random
from fractions import Fraction

import numpy as np
import pytest

import bruteforce
import gen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                key, val = line.split()
                out[key] = val
    return out


# ---------------------------------------------------------------- constants

def test_rho_half_range_from_paper_discretisation():
    g = read_golden("paper_discretization.txt")
    rho_max_mm = Fraction(g["rho_max"])
    assert Fraction(g["rho_min"]) == -rho_max_mm
    # fixed point: u_q has scale 2^32 per um^-1, trig 2^14, so rho_q has 2^46 per um^-1
    h = round(rho_max_mm / 1000 * 2 ** 46)
    assert oracle.const_H() == h == 703687442
    # the paper's bin width: 2 rho_max / bins == delta rho
    assert 2 * rho_max_mm / int(g["rho_bins"]) == Fraction(g["delta_rho"])
    # and in fixed point, one of the 1000 bins spans 2H/1000 units == delta rho * 2^46 / 1000 (to rounding)
    assert abs(Fraction(2 * h, 1000) - Fraction(g["delta_rho"]) / 1000 * 2 ** 46) < 1


def test_bin_edges_match_paper_equal_width_bins():
    """rho bin k of N covers [-0.01 + k d, -0.01 + (k+1) d) mm^-1 with d = 0.02/N (Sec. 2)."""
    g = read_golden("paper_discretization.txt")
    rmin, rmax = Fraction(g["rho_min"]), Fraction(g["rho_max"])
    for n_rho in (int(g["rho_bins"]), 64, 256, 512):
        d = (rmax - rmin) / n_rho
        for k in list(range(0, n_rho, max(1, n_rho // 37))) + [n_rho - 1]:
            lo = (rmin + k * d) / 1000 * 2 ** 46  # edge in fixed-point units (exact rational)
            hi = (rmin + (k + 1) * d) / 1000 * 2 ** 46
            # well inside the bin (edges move by < 1 unit because H is rounded)
            assert oracle.bin_of(math.ceil(lo) + 2, n_rho) == k
            assert oracle.bin_of(math.floor(hi) - 2, n_rho) == k
            if k > 0:
                assert oracle.bin_of(math.floor(lo) - 2, n_rho) == k - 1
    # out-of-range rho is clamped to the edge bins
    assert oracle.bin_of(-10 ** 12, 256) == 0
    assert oracle.bin_of(10 ** 12, 256) == 255


def test_trig_tables_bin_centres():
    for n in (4, 64, 256, 512, 1000, 1024):
        c, s = oracle.tables(n)
        c = c.astype(np.int64)
        s = s.astype(np.int64)
        # centres are symmetric about pi/2: th_{N-1-j} = pi - th_j
        assert np.array_equal(c[::-1], -c)
        assert np.array_equal(s[::-1], s)
        assert np.all(np.abs(c * c + s * s - 2 ** 28) <= 2 * 16384)
        j = n // 3
        th = (j + 0.5) * math.pi / n
        assert c[j] == round(16384 * math.cos(th)) and s[j] == round(16384 * math.sin(th))


def test_trig_rounding_never_near_half():
    """The tables are rounded from doubles; no entry lies within 1e-7 of a .5 tie for any
    N_theta in [4, 1024], so any correctly computed cos/sin gives the same table."""
    worst = 1.0
    for n in range(4, 1025):
        th = (np.arange(n) + 0.5) * math.pi / n
        for v in (16384 * np.cos(th), 16384 * np.sin(th)):
            f = np.abs(v) - np.floor(np.abs(v))
            worst = min(worst, float(np.min(np.abs(f - 0.5))))
    assert worst > 1e-7


def test_checksum_hash_is_published_splitmix64_finaliser():
    mask = (1 << 64) - 1

    def fin(z):
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        return z ^ (z >> 31)

    for key, val in read_golden("splitmix64_seed0.txt").items():
        assert fin(int(key) * 0x9E3779B97F4A7C15 & mask) == int(val, 16)
    acc = np.zeros((8, 8), np.int16)
    acc[2, 5] = 7
    assert oracle.checksum(acc) == (7 * fin(2 * 8 + 5 + 1)) & mask
    acc[7, 7] = 3
    assert oracle.checksum(acc) == (7 * fin(22) + 3 * fin(64)) & mask


# ---------------------------------------------------------------- map (Eq. 1-2)

def test_map_circle_through_origin_becomes_line():
    """A circle through the origin with centre (a, b) satisfies x^2 + y^2 = 2ax + 2by, so
    u = 2x/r^2, v = 2y/r^2 lie on a u + b v = 1 (the line of Eq. 2 with th = atan2(b,a),
    rho = 1/R)."""
    rng = random.Random(7)
    for _ in range(200):
        a = rng.uniform(-900.0, 900.0) * 1000
        b = rng.uniform(-900.0, 900.0) * 1000
        R = math.hypot(a, b)
        phic = math.atan2(b, a)
        r = rng.uniform(200e3, min(2 * R, 811e3)) if 2 * R > 200e3 else None
        if r is None:
            continue
        phi = phic + rng.choice((-1, 1)) * math.acos(r / (2 * R))
        x, y = round(r * math.cos(phi)), round(r * math.sin(phi))
        st, u, v = oracle.map_hit(x, y)
        assert st == 0
        lhs = (a * u + b * v) / 2 ** 32
        # u_q floors (1 unit) and the hit is rounded to 1 um: relative error well below 1e-3
        assert abs(lhs - 1.0) < 1e-3


def test_map_floor_semantics_and_bad_hits():
    # u = 2x/r^2 rounded toward -infinity, for both signs
    st, u, v = oracle.map_hit(200000, 0)
    assert (st, u, v) == (0, 42949, 0)  # 2^33 / 2e5 = 42949.67...
    st, u, v = oracle.map_hit(-200000, 0)
    assert (st, u, v) == (0, -42950, 0)
    st, u, v = oracle.map_hit(0, -200000)
    assert (st, u, v) == (0, 0, -42950)
    assert oracle.map_hit(0, 0)[0] == oracle.F_BAD_HIT
    assert oracle.map_hit(2 ** 24 + 1, 5)[0] == oracle.F_BAD_HIT
    assert oracle.map_hit(5, -(2 ** 24) - 1)[0] == oracle.F_BAD_HIT
    assert oracle.map_hit(2 ** 24, -(2 ** 24))[0] == 0


# ---------------------------------------------------------------- P1 closed form

def circle_hits(xc_mm, yc_mm):
    """Hits on the exact circle through the origin with centre (xc, yc), one per layer radius
    200 + 13 l mm it reaches (outgoing side), rounded to um."""
    R = math.hypot(xc_mm, yc_mm)
    phic = math.atan2(yc_mm, xc_mm)
    hits = []
    for l in range(48):
        r = 200.0 + 13.0 * l
        if r > 2 * R:
            break
        phi = phic + math.acos(r / (2 * R))
        hits.append((round(1000 * r * math.cos(phi)), round(1000 * r * math.sin(phi))))
    return hits


@pytest.mark.parametrize("n_theta,n_rho,j,k", [
    (256, 256, 75, 153), (256, 256, 0, 200), (256, 256, 255, 60), (256, 256, 128, 40),
    (64, 64, 10, 45), (512, 512, 300, 100), (1000, 1000, 777, 888), (256, 256, 31, 127)])
def test_p1_single_track_peaks_at_closed_form_cell(n_theta, n_rho, j, k):
    """Eq. (2): the line u cos th + v sin th = rho is the circle with centre (cos th / rho,
    sin th / rho). Put th at the centre of column j and rho at the centre of rho bin k: every
    hit of that circle must vote in cell (j, k), which must be a peak, and every hit kept."""
    th = (j + 0.5) * math.pi / n_theta
    rho = -0.01 + (k + 0.5) * 0.02 / n_rho
    if abs(rho) > 0.0085:
        pytest.skip("circle too small for the chamber")
    hits = circle_hits(math.cos(th) / rho, math.sin(th) / rho)
    assert len(hits) >= 3
    xy = np.array(hits, np.int32)
    off = np.array([0, len(hits)], np.int64)
    p = oracle.params(n_theta, n_rho, 2)
    r = oracle.run(xy, off, p, with_acc=True)
    acc = r.acc[0]
    assert acc[j, k] == len(hits)
    assert int(np.argmax(acc)) == j * n_rho + k
    stored = r.peaks[0][: r.npeaks[0]]
    assert any(int(q["theta_bin"]) == j and int(q["rho_bin"]) == k and int(q["votes"]) == len(hits) for q in stored)
    assert r.mask.sum() == len(hits) and r.nkept[0] == len(hits)
    # every column holds exactly one vote per hit
    assert np.all(acc.sum(axis=1) == len(hits))


def test_p1_random_circles_peak_near_closed_form():
    rng = random.Random(11)
    n = 256
    dth, drho = math.pi / n, 0.02 / n
    for _ in range(40):
        R = rng.uniform(130.0, 2000.0)
        phic = rng.uniform(-math.pi, math.pi)
        xc, yc = R * math.cos(phic), R * math.sin(phic)
        hits = circle_hits(xc, yc)
        if len(hits) < 4:
            continue
        th, rho = math.atan2(yc, xc), 1.0 / R
        if th < 0:
            th, rho = th + math.pi, -rho
        ej, ek = int(th // dth), int((rho + 0.01) // drho)
        r = oracle.run(np.array(hits, np.int32), np.array([0, len(hits)], np.int64), oracle.params(n, n, 2),
                       with_acc=True)
        aj, ak = divmod(int(np.argmax(r.acc[0])), n)
        dj = min(abs(aj - ej), n - abs(aj - ej))
        assert dj <= 1 and abs(ak - ek) <= 1 or (dj <= 1 and abs((n - 1 - ak) - ek) <= 1 and (aj == 0 or aj == n - 1))


# ---------------------------------------------------------------- Eq. (2) circle recovery

@pytest.mark.parametrize("n_theta,n_rho,j,k", [(256, 256, 75, 153), (256, 256, 255, 60), (512, 512, 300, 100),
                                               (1000, 1000, 777, 888), (64, 64, 10, 45)])
def test_circle_of_the_peak_passes_through_the_hits(n_theta, n_rho, j, k):
    """The circle that a track's peak stands for (Eq. 2 at the bin centres) must pass through
    the track's hits (to their 1 um rounding) and through the origin."""
    th = (j + 0.5) * math.pi / n_theta
    rho = -0.01 + (k + 0.5) * 0.02 / n_rho
    if abs(rho) > 0.0085:
        pytest.skip("circle too small for the chamber")
    hits = circle_hits(math.cos(th) / rho, math.sin(th) / rho)
    r = oracle.run(np.array(hits, np.int32), np.array([0, len(hits)], np.int64), oracle.params(n_theta, n_rho, 2))
    stored = r.peaks[0][: r.npeaks[0]]
    mine = [q for q in stored if int(q["theta_bin"]) == j and int(q["rho_bin"]) == k]
    assert len(mine) == 1
    xc, yc, rc, pt = oracle.circles(np.array(mine), n_theta, n_rho)[0]
    assert abs(math.hypot(xc, yc) - rc) < 1e-9 * rc                      # through the origin
    for (x, y) in hits:                                                  # through every hit
        assert abs(math.hypot(x / 1000.0 - xc, y / 1000.0 - yc) - rc) < 2e-3
    assert abs(pt - 0.3 * rc) < 1e-9 * pt                                # 1 T


def test_circles_of_random_tracks_within_one_bin():
    """Random circles through the origin: the accumulator maximum's circle has 1/r_c within
    1.5 rho-bins of the true curvature and its centre direction within 1.5 theta-bins."""
    rng = random.Random(5)
    n = 256
    dth, drho = math.pi / n, 0.02 / n
    checked = 0
    for _ in range(60):
        R = rng.uniform(130.0, 2000.0)
        phic = rng.uniform(-math.pi, math.pi)
        hits = circle_hits(R * math.cos(phic), R * math.sin(phic))
        if len(hits) < 6:
            continue
        r = oracle.run(np.array(hits, np.int32), np.array([0, len(hits)], np.int64), oracle.params(n, n, 2),
                       with_acc=True)
        aj, ak = divmod(int(np.argmax(r.acc[0])), n)
        pk = np.zeros(1, oracle.PEAK_DTYPE)
        pk["theta_bin"], pk["rho_bin"] = aj, ak
        xc, yc, rc, pt = oracle.circles(pk, n, n)[0]
        assert abs(1.0 / rc - 1.0 / R) <= 1.5 * drho
        d = math.atan2(yc, xc) - phic
        d = (d + math.pi) % (2 * math.pi) - math.pi
        assert abs(d) <= 1.5 * dth
        checked += 1
    assert checked > 30


def test_circle_sign_convention():
    """rho < 0 stands for the circle whose centre lies opposite the column's normal (theta + pi);
    a bin centre at rho = 0 (odd N_rho) is the straight line, radius infinite."""
    pk = np.zeros(3, oracle.PEAK_DTYPE)
    pk["theta_bin"] = [0, 0, 0]
    pk["rho_bin"] = [0, 4, 2]
    out = oracle.circles(pk, 4, 5)
    assert out[0][0] < 0 and out[0][1] < 0 and out[1][0] > 0 and out[1][1] > 0
    assert np.allclose(out[0][:3], -out[1][:3] * np.array([1, 1, -1]))
    assert math.isinf(out[2][2]) and math.isinf(out[2][3])


# ---------------------------------------------------------------- P2 invariants

def local_max_rule(acc, T):
    """Numpy form of the 3x3 peak rule (independent of the oracle's loops)."""
    nt, nr = acc.shape
    a = acc.astype(np.int32)
    pad = np.full((nt + 2, nr + 2), -1, np.int32)
    pad[1:-1, 1:-1] = a
    pad[0, 1:-1] = a[-1, ::-1]  # column -1 = column nt-1 mirrored
    pad[-1, 1:-1] = a[0, ::-1]  # column nt = column 0 mirrored
    ok = a >= T
    for dj in (-1, 0, 1):
        for dk in (-1, 0, 1):
            if dj == 0 and dk == 0:
                continue
            b = pad[1 + dj:1 + dj + nt, 1 + dk:1 + dk + nr]
            if dj == 0:
                prec = np.full((nt, nr), dk < 0)
            elif dj == -1:
                prec = np.ones((nt, nr), bool)
                prec[0, :] = False  # the wrapped column nt-1 follows column 0
            else:
                prec = np.zeros((nt, nr), bool)
                prec[-1, :] = True  # the wrapped column 0 precedes column nt-1
            ok &= np.where(b < 0, True, np.where(prec, a > b, a >= b))
    return ok


@pytest.mark.parametrize("name,n", [("plain_small", 100), ("plain_paper", 12), ("stress", 2)])
def test_p2_invariants(name, n):
    cfg = gen.CONFIGS[name]
    ev = gen.generate(cfg, n)
    p = oracle.params(cfg.n_theta, cfg.n_rho, cfg.threshold, max_peaks=1 << 14)
    r = oracle.run(ev.xy, ev.off, p, with_acc=True, threads=4)
    assert r.status == 0
    tab = bruteforce.trig(cfg.n_theta)
    for e in range(ev.n_events):
        a, b = ev.off[e], ev.off[e + 1]
        acc = r.acc[e]
        assert np.all(acc.sum(axis=1) == b - a)
        rule = local_max_rule(acc, cfg.threshold)
        js, ks = np.nonzero(rule)
        stored = r.peaks[e][: r.npeaks[e]]
        assert r.npeaks[e] == len(js)
        assert np.array_equal(stored["theta_bin"], js) and np.array_equal(stored["rho_bin"], ks)
        assert np.array_equal(stored["votes"], acc[js, ks])
        assert r.nkept[e] == r.mask[a:b].sum()
        if e < 3:  # witnesses, with the independent restatement's arithmetic
            cols = {}
            for q in stored:
                cols.setdefault(int(q["theta_bin"]), []).append(int(q["rho_bin"]))
            for i in range(a, b):
                u, v = bruteforce.conformal(int(ev.xy[i, 0]), int(ev.xy[i, 1]))
                hit = any(abs(bruteforce.rho_bin(u, v, *tab[j], cfg.n_rho) - k) <= 1
                          for j, ks_ in cols.items() for k in ks_)
                assert r.mask[i] == hit


# ---------------------------------------------------------------- P3 brute force

def test_p3_bruteforce_tiny_events():
    rng = random.Random(3)
    for trial in range(120):
        n_theta = rng.choice((4, 8, 16))
        n_rho = rng.choice((4, 8, 16))
        T = rng.choice((1, 2, 3))
        nh = rng.randint(0, 20)
        hits = []
        for _ in range(nh):
            kind = rng.random()
            if kind < 0.05:
                hits.append((0, 0))
            elif kind < 0.25:  # small radii: rho far out of range, clamped
                hits.append((rng.randint(-3000, 3000), rng.randint(-3000, 3000)))
            else:
                r = rng.uniform(150e3, 900e3)
                phi = rng.uniform(0, 2 * math.pi)
                hits.append((round(r * math.cos(phi)), round(r * math.sin(phi))))
        maxp = rng.choice((1, 3, 64))
        acc_b, peaks_b, mask_b = bruteforce.event(hits, n_theta, n_rho, T, 1, maxp)
        xy = np.array(hits, np.int32).reshape(-1, 2)
        r = oracle.run(xy, np.array([0, nh], np.int64), oracle.params(n_theta, n_rho, T, 1, maxp), with_acc=True)
        dense = np.zeros((n_theta, n_rho), np.int16)
        for (j, k), vv in acc_b.items():
            dense[j, k] = vv
        assert np.array_equal(r.acc[0], dense), trial
        assert r.npeaks[0] == len(peaks_b)
        stored = r.peaks[0][: min(r.npeaks[0], maxp)]
        assert [(int(q["theta_bin"]), int(q["rho_bin"]), int(q["votes"])) for q in stored] == peaks_b[:maxp]
        assert list(r.mask) == mask_b
        bad = sum(1 for h in hits if h == (0, 0))
        assert (r.status & oracle.F_BAD_HIT) == (oracle.F_BAD_HIT if bad else 0)
        assert ((r.status & oracle.F_PEAK_OVERFLOW) != 0) == (len(peaks_b) > maxp)


# ---------------------------------------------------------------- P5 hand cases

def peaks_of(cells, T=2, nt=8, nr=8, maxp=64):
    acc = np.zeros((nt, nr), np.int16)
    for (j, k), v in cells.items():
        acc[j, k] = v
    n, st = oracle.peaks(acc, oracle.params(nt, nr, T, 1, maxp))
    return n, [(int(q["theta_bin"]), int(q["rho_bin"]), int(q["votes"])) for q in st]


def test_p5_single_and_threshold():
    assert peaks_of({(3, 3): 5}) == (1, [(3, 3, 5)])
    assert peaks_of({(3, 3): 1}) == (0, [])
    assert peaks_of({(3, 3): 2}) == (1, [(3, 3, 2)])


def test_p5_plateaus():
    assert peaks_of({(3, 3): 5, (3, 4): 5}) == (1, [(3, 3, 5)])  # along rho
    assert peaks_of({(3, 3): 5, (4, 3): 5}) == (1, [(3, 3, 5)])  # along theta
    assert peaks_of({(3, 3): 5, (4, 4): 5}) == (1, [(3, 3, 5)])  # diagonal
    assert peaks_of({(3, 4): 5, (4, 3): 5}) == (1, [(3, 4, 5)])  # anti-diagonal
    assert peaks_of({(3, 3): 5, (3, 4): 5, (4, 3): 5}) == (1, [(3, 3, 5)])  # L of three
    # a V-shaped plateau whose arms do not touch yields one peak per arm start
    assert peaks_of({(2, 2): 5, (3, 3): 5, (2, 4): 5}) == (2, [(2, 2, 5), (2, 4, 5)])
    # a higher neighbour suppresses
    assert peaks_of({(3, 3): 5, (3, 4): 6}) == (1, [(3, 4, 6)])
    assert peaks_of({(3, 3): 5, (2, 2): 6}) == (1, [(2, 2, 6)])


def test_p5_theta_wrap_mirrors_rho():
    # column -1 of (0, 2) is column 7 at rho 7-2 = 5; (7, 5) follows (0, 2) in raster order
    assert peaks_of({(0, 2): 5, (7, 5): 5}) == (1, [(0, 2, 5)])
    assert peaks_of({(0, 2): 5, (7, 5): 6}) == (1, [(7, 5, 6)])
    assert peaks_of({(0, 2): 6, (7, 5): 5}) == (1, [(0, 2, 6)])
    # mirrored diagonal neighbours: (0, 2) touches (7, 4), (7, 5), (7, 6)
    assert peaks_of({(0, 2): 5, (7, 4): 5}) == (1, [(0, 2, 5)])
    assert peaks_of({(0, 2): 5, (7, 6): 7}) == (1, [(7, 6, 7)])
    # not mirrored: (7, 2) is no neighbour of (0, 2)
    assert peaks_of({(0, 2): 5, (7, 2): 5}) == (2, [(0, 2, 5), (7, 2, 5)])


def test_p5_rho_edges():
    assert peaks_of({(3, 0): 5}) == (1, [(3, 0, 5)])
    assert peaks_of({(3, 7): 5}) == (1, [(3, 7, 5)])
    assert peaks_of({(3, 7): 5, (4, 7): 5}) == (1, [(3, 7, 5)])
    # corner with wrap: (0, 0)'s wrapped neighbours are (7, 7) and (7, 6)
    assert peaks_of({(0, 0): 5, (7, 7): 5}) == (1, [(0, 0, 5)])
    assert peaks_of({(0, 0): 5, (7, 6): 5}) == (1, [(0, 0, 5)])
    assert peaks_of({(0, 7): 5, (7, 0): 5}) == (1, [(0, 7, 5)])


def test_p5_overflow_keeps_raster_order():
    cells = {(1, 1): 3, (1, 5): 4, (4, 2): 9, (6, 6): 2}
    assert peaks_of(cells, maxp=2) == (4, [(1, 1, 3), (1, 5, 4)])
    assert peaks_of(cells, maxp=4)[1] == [(1, 1, 3), (1, 5, 4), (4, 2, 9), (6, 6, 2)]


def test_p5_overflow_limits_selection():
    """Only stored peaks select hits: with max_peaks = 1 only the first (raster) track is kept."""
    n = 64
    hits, parts = [], []
    for (j, k) in ((10, 40), (50, 20)):
        th = (j + 0.5) * math.pi / n
        rho = -0.01 + (k + 0.5) * 0.02 / n
        h = circle_hits(math.cos(th) / rho, math.sin(th) / rho)
        parts.append(len(h))
        hits += h
    xy = np.array(hits, np.int32)
    off = np.array([0, len(hits)], np.int64)
    full = oracle.run(xy, off, oracle.params(n, n, 6, 0, 64))
    one = oracle.run(xy, off, oracle.params(n, n, 6, 0, 1))
    assert full.npeaks[0] == one.npeaks[0] >= 2
    assert one.status & oracle.F_PEAK_OVERFLOW and not full.status & oracle.F_PEAK_OVERFLOW
    assert one.mask[: parts[0]].all() and one.nkept[0] < full.nkept[0]


# ---------------------------------------------------------------- P6 permutation

def test_p6_permutation_invariance():
    cfg = gen.CONFIGS["plain_small"]
    ev = gen.generate(cfg, 5)
    p = oracle.params(cfg.n_theta, cfg.n_rho, cfg.threshold)
    rng = np.random.default_rng(5)
    for e in range(5):
        a, b = ev.off[e], ev.off[e + 1]
        xy = ev.xy[a:b]
        perm = rng.permutation(b - a)
        r1 = oracle.run(xy, np.array([0, b - a]), p, with_acc=True)
        r2 = oracle.run(xy[perm], np.array([0, b - a]), p, with_acc=True)
        assert np.array_equal(r1.acc, r2.acc)
        assert np.array_equal(r1.peaks, r2.peaks) and np.array_equal(r1.npeaks, r2.npeaks)
        assert np.array_equal(r1.mask[perm], r2.mask)


# ---------------------------------------------------------------- batch driver, metrics

def test_offsets_validation_and_threads():
    cfg = gen.CONFIGS["plain_small"]
    ev = gen.generate(cfg, 20)
    p = oracle.params(cfg.n_theta, cfg.n_rho, cfg.threshold)
    r1 = oracle.run(ev.xy, ev.off, p, threads=1)
    r4 = oracle.run(ev.xy, ev.off, p, threads=4)
    assert np.array_equal(r1.mask, r4.mask) and np.array_equal(r1.checksum, r4.checksum)
    bad = ev.off.copy()
    bad[5], bad[6] = bad[6], bad[5]
    assert oracle.run(ev.xy, bad, p).status == oracle.F_BAD_OFFSETS
    bad = ev.off.copy()
    bad[-1] -= 1
    assert oracle.run(ev.xy, bad, p).status == oracle.F_BAD_OFFSETS


def test_event_too_large_is_skipped():
    xy = np.tile(np.array([[250000, 1000]], np.int32), (32768, 1))
    r = oracle.run(xy, np.array([0, 32768]), oracle.params(8, 8, 1), with_acc=True)
    assert r.status == oracle.F_EVENT_TOO_LARGE
    assert r.npeaks[0] == 0 and r.nkept[0] == 0 and r.acc.sum() == 0


def test_metrics_eq8_eq9():
    mask = np.array([1, 0, 1, 1, 0], np.uint8)
    truth = np.array([0, -1, -1, 1, 2], np.int32)
    rc, rs = oracle.metrics(mask, truth)
    assert rc == pytest.approx(3 / 5)  # N_select / N_total
    assert rs == pytest.approx(2 / 3)  # N_true,select / N_true


# ---------------------------------------------------------------- iterative peak finder (Sec. 2)

def _in_window(a, b, R, NT, NR):
    """Is cell b within the suppression window of cell a (theta wrap with mirrored rho)?"""
    (ja, ka), (jb, kb) = a, b
    for dj in range(-R, R + 1):
        jj = ja + dj
        mirrored = jj < 0 or jj >= NT
        jj %= NT
        if jj != jb:
            continue
        for dk in range(-R, R + 1):
            kk = ka + dk
            if kk < 0 or kk >= NR:
                continue
            if (NR - 1 - kk if mirrored else kk) == kb:
                return True
    return False


def _greedy_peaks(acc, T, num, den, R):
    """Independent restatement: candidates sorted by (votes desc, raster asc), each accepted
    unless it lies in the window of an accepted one."""
    NT, NR = acc.shape
    amax = int(acc.max()) if acc.size else 0
    cand = [(-int(acc[j, k]), j * NR + k) for j in range(NT) for k in range(NR)
            if acc[j, k] >= T and int(acc[j, k]) * den >= num * amax]
    out = []
    for negv, c in sorted(cand):
        cell = divmod(c, NR)
        if not any(_in_window(p, cell, R, NT, NR) for p, _ in out):
            out.append((cell, -negv))
    return out


@pytest.mark.parametrize("seed", range(12))
def test_iterative_matches_greedy_restatement(seed):
    rng = np.random.default_rng(seed)
    NT, NR = int(rng.choice([4, 6, 8, 9])), int(rng.choice([4, 5, 8, 11]))
    acc = rng.integers(0, 9, size=(NT, NR)).astype(np.int16)
    T, num, den, R = int(rng.integers(1, 4)), int(rng.integers(0, 3)), 4, int(rng.integers(0, 3))
    p = oracle.params(NT, NR, T, 1, 1000, peak_mode=oracle.PEAK_ITERATIVE, rel_num=num, rel_den=den, nms_radius=R)
    n, pk = oracle.peaks_iterative(acc, p)
    exp = _greedy_peaks(acc, T, num, den, R)
    assert n == len(exp)
    assert [((int(q["theta_bin"]), int(q["rho_bin"])), int(q["votes"])) for q in pk] == exp


def _rounds_peaks(acc, T, num, den, R, push=False, order_rng=None, window_max_round0=False):
    """The kept set reached by rounds of local rules (no ordering of the work): a candidate
    (cell passing the thresholds) is dropped once a kept candidate lies in its window, and kept
    once every higher-ranked candidate in its window is dropped; rank is (votes desc, raster
    asc). Each round applies the rules to every undecided candidate on the states of the round
    before. With push, a candidate kept in a round also drops every undecided candidate of its
    window at once. With order_rng, a round visits the candidates in a random order and each
    decision (and push) is seen by the visits after it (the GPU's threads read states while
    others change them). With window_max_round0, round 0 keeps exactly the candidates whose
    window holds no cell of more votes (ties by raster order), read from the votes alone, and
    pushes their drops: the GPU's round 0. The kept cells, listed in rank order."""
    NT, NR = acc.shape
    amax = int(acc.max()) if acc.size else 0
    cand = [(j, k) for j in range(NT) for k in range(NR) if acc[j, k] >= T and int(acc[j, k]) * den >= num * amax]
    rank = {c: (-int(acc[c]), c[0] * NR + c[1]) for c in cand}
    window = {c: [d for d in cand if d != c and _in_window(c, d, R, NT, NR)] for c in cand}
    state = {c: 0 for c in cand}  # 0 undecided, 1 dropped, 2 kept
    if window_max_round0:
        cells = [(j, k) for j in range(NT) for k in range(NR)]
        rank_all = {c: (-int(acc[c]), c[0] * NR + c[1]) for c in cells}
        top = [c for c in cand if all(rank_all[d] > rank_all[c] for d in cells if d != c and _in_window(c, d, R, NT, NR))]
        for c in top:
            state[c] = 2
        for c in top:
            for d in window[c]:
                assert state[d] != 2
                state[d] = 1
    for _ in range(len(cand) + 1):
        new = dict(state)
        seen = new if order_rng is not None else state  # in place: later visits see earlier ones
        visit = list(cand) if order_rng is None else [cand[i] for i in order_rng.permutation(len(cand))]
        for c in visit:
            if seen[c]:
                continue
            if any(seen[d] == 2 for d in window[c]):
                new[c] = 1
            elif all(seen[d] == 1 for d in window[c] if rank[d] < rank[c]):
                new[c] = 2
                if push:
                    for d in window[c]:
                        assert new[d] != 2, "a kept cell never lies in the window of one kept later"
                        if new[d] == 0:
                            new[d] = 1
        if new == state:
            break
        state = new
    assert all(state.values()), "every candidate is decided"
    kept = sorted((c for c in cand if state[c] == 2), key=lambda c: rank[c])
    return [(c, int(acc[c])) for c in kept]


@pytest.mark.parametrize("seed", range(16))
def test_iterative_local_rules_reach_the_greedy_list(seed):
    """The GPU decides the kept set by the local rules of _rounds_peaks (a kept cell in the
    window of an undecided candidate drops it; a candidate whose higher-ranked window cells are
    all dropped is kept). The window relation is symmetric (checked here too), so these rules
    reach exactly the oracle's extraction list, ties and theta wrap included."""
    rng = np.random.default_rng(100 + seed)
    NT, NR = int(rng.choice([4, 6, 8, 12])), int(rng.choice([4, 5, 8, 11]))
    acc = rng.integers(0, int(rng.choice([3, 6, 12])), size=(NT, NR)).astype(np.int16)
    T, num, den = int(rng.integers(1, 3)), int(rng.integers(0, 3)), 4
    R = int(rng.integers(0, (NT - 1) // 2 + 1))
    cells = [(j, k) for j in range(NT) for k in range(NR)]
    for a in cells[::3]:
        for b in cells[::2]:
            assert _in_window(a, b, R, NT, NR) == _in_window(b, a, R, NT, NR)
    p = oracle.params(NT, NR, T, 1, 1000, peak_mode=oracle.PEAK_ITERATIVE, rel_num=num, rel_den=den, nms_radius=R)
    n, pk = oracle.peaks_iterative(acc, p)
    exp = [((int(q["theta_bin"]), int(q["rho_bin"])), int(q["votes"])) for q in pk]
    # synchronous rounds, with and without pushed drops, and in-place rounds in random orders
    for push, order, w0 in ((False, None, False), (True, None, False), (True, np.random.default_rng(seed), False),
                            (False, np.random.default_rng(50 + seed), False), (True, np.random.default_rng(seed), True)):
        got = _rounds_peaks(acc, T, num, den, R, push=push, order_rng=order, window_max_round0=w0)
        assert n == len(got)
        assert exp == got, (push, order is not None)


def test_iterative_hand_cases():
    NT, NR = 8, 8
    acc = np.zeros((NT, NR), np.int16)
    acc[2, 3] = 20      # the maximum
    acc[3, 4] = 19      # its diagonal neighbour: suppressed with R = 1, extracted with R = 0
    acc[6, 1] = 10      # exactly half the maximum: qualifies at 1/2 (10 * 2 >= 1 * 20)
    acc[5, 6] = 9       # below half
    acc[0, 0] = 15      # column 0 ...
    acc[7, 6] = 15      # ... its wrapped neighbour (column -1 = 7, row 8-1-(0+1) = 6): tie, follows
    p = lambda R, num, den, mx=100: oracle.params(NT, NR, 1, 1, mx, peak_mode=1, rel_num=num, rel_den=den,
                                                 nms_radius=R)
    n, pk = oracle.peaks_iterative(acc, p(1, 1, 2))
    got = [(int(q["theta_bin"]), int(q["rho_bin"]), int(q["votes"])) for q in pk]
    assert got == [(2, 3, 20), (0, 0, 15), (6, 1, 10)]
    n, pk = oracle.peaks_iterative(acc, p(0, 1, 2))
    got = [(int(q["theta_bin"]), int(q["rho_bin"]), int(q["votes"])) for q in pk]
    assert got == [(2, 3, 20), (3, 4, 19), (0, 0, 15), (7, 6, 15), (6, 1, 10)]
    n, pk = oracle.peaks_iterative(acc, p(1, 0, 1))       # no relative cut: the 9 is found too
    assert n == 4 and int(pk[-1]["votes"]) == 9
    n, pk = oracle.peaks_iterative(acc, p(0, 1, 2, mx=2))  # overflow: the true count, two stored
    assert n == 5 and len(pk) == 2


def test_iterative_invariants_on_events():
    """On real events: every peak qualifies, no peak lies in another's window, and every
    qualifying cell lies in the window of a peak extracted before it would have been."""
    cfg = gen.CONFIGS["plain_paper"]
    ev = gen.generate(cfg, 6)
    NT = NR = 64
    p = oracle.params(NT, NR, 6, 1, 4096, peak_mode=1, rel_num=1, rel_den=3, nms_radius=2)
    r = oracle.run(ev.xy, ev.off, p, with_acc=True)
    for e in range(ev.n_events):
        acc = r.acc[e].astype(np.int64)
        amax = int(acc.max())
        peaks = [((int(q["theta_bin"]), int(q["rho_bin"])), int(q["votes"])) for q in r.peaks[e][: r.npeaks[e]]]
        assert len(peaks) == r.npeaks[e] > 0
        for (c, v) in peaks:
            assert v == acc[c] and v >= 6 and 3 * v >= amax
        for a in range(len(peaks)):
            for b in range(len(peaks)):
                if a != b:
                    assert not _in_window(peaks[a][0], peaks[b][0], 2, NT, NR)
        order = {c: (-v, c[0] * NR + c[1]) for c, v in peaks}
        for j in range(NT):
            for k in range(NR):
                v = int(acc[j, k])
                if v < 6 or 3 * v < amax or (j, k) in order:
                    continue
                assert any(_in_window(c, (j, k), 2, NT, NR) and order[c] < (-v, j * NR + k) for c, _ in peaks)
