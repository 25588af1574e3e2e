"""Independent big-integer restatement of the method, for tiny events.

Written separately from the C oracle (no shared code): Python integers, ``//``
floor semantics, dictionaries instead of arrays. Used to cross-check the oracle
exhaustively on events of a few hits and accumulators of 4..16 bins a side.
"""
from fractions import Fraction
import math

# rho half-range: 0.01 mm^-1 = 1e-5 um^-1, in units of 2^-46 um^-1, rounded to nearest
H = round(Fraction(1, 100000) * 2 ** 46)


def round_half_away(x: float) -> int:
    return int(math.floor(x + 0.5)) if x >= 0 else -int(math.floor(-x + 0.5))


def trig(n_theta: int):
    out = []
    for j in range(n_theta):
        th = (j + 0.5) * math.pi / n_theta
        out.append((round_half_away(16384 * math.cos(th)), round_half_away(16384 * math.sin(th))))
    return out


def conformal(x: int, y: int):
    if abs(x) > 2 ** 24 or abs(y) > 2 ** 24:
        return None
    r2 = x * x + y * y
    if r2 == 0:
        return None
    return (2 * x * 2 ** 32) // r2, (2 * y * 2 ** 32) // r2


def rho_bin(u: int, v: int, c: int, s: int, n_rho: int) -> int:
    t = u * c + v * s + H
    if t < 0:
        return 0
    return min(n_rho - 1, (t * n_rho) // (2 * H))


def neighbours(j: int, k: int, n_theta: int, n_rho: int):
    for dj in (-1, 0, 1):
        for dk in (-1, 0, 1):
            if dj == 0 and dk == 0:
                continue
            jj, kk = j + dj, k + dk
            if not 0 <= kk < n_rho:
                continue
            if jj < 0 or jj >= n_theta:
                jj %= n_theta
                kk = n_rho - 1 - kk
            yield jj, kk


def event(hits, n_theta, n_rho, threshold, keep_halfwidth=1, max_peaks=1024):
    """Returns (acc dict {(j,k): votes}, peaks [(j,k,votes)] (all), mask [0/1])."""
    tab = trig(n_theta)
    mapped = [conformal(x, y) for x, y in hits]
    acc = {}
    for m in mapped:
        if m is None:
            continue
        for j, (c, s) in enumerate(tab):
            key = (j, rho_bin(m[0], m[1], c, s, n_rho))
            acc[key] = acc.get(key, 0) + 1
    peaks = []
    for j in range(n_theta):
        for k in range(n_rho):
            a = acc.get((j, k), 0)
            if a < threshold:
                continue
            me = j * n_rho + k
            ok = True
            for jj, kk in neighbours(j, k, n_theta, n_rho):
                b = acc.get((jj, kk), 0)
                if jj * n_rho + kk < me:
                    ok = ok and a > b
                else:
                    ok = ok and a >= b
            if ok:
                peaks.append((j, k, a))
    stored = peaks[:max_peaks]
    mask = []
    for m in mapped:
        keep = 0
        if m is not None:
            for j, k, _ in stored:
                c, s = tab[j]
                if abs(rho_bin(m[0], m[1], c, s, n_rho) - k) <= keep_halfwidth:
                    keep = 1
                    break
        mask.append(keep)
    return acc, peaks, mask
