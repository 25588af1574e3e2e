"""Run as a child process by test_phase_timers.py: the phase-timer build of the library gives
the oracle's results (counts, peak records, masks) on a small batch and counts cycles in the
phases that ran."""
import json
import os
import sys

os.environ["HOUGH_PHASE_TIMERS"] = "1"
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import numpy as np  # noqa: E402
import torch  # noqa: E402

import gen  # noqa: E402
import oracle  # noqa: E402
import paper_2607_04067_gb300 as h  # noqa: E402


def main():
    mode = int(sys.argv[1])
    cfg = gen.CONFIGS["plain_paper"]
    ev = gen.generate(cfg, 64)
    kw = dict(peak_mode=mode, rel_num=1, rel_den=2, nms_radius=3) if mode else {}
    op = oracle.params(cfg.n_theta, cfg.n_rho, cfg.threshold, cfg.keep_halfwidth, 512, **kw)
    ref = oracle.run(ev.xy, ev.off, op, threads=os.cpu_count() or 1)
    p = h.params(cfg.n_theta, cfg.n_rho, cfg.threshold, cfg.keep_halfwidth, 512, **kw)
    xy, off = torch.from_numpy(ev.xy).cuda(), torch.from_numpy(ev.off).cuda()
    h.phase_cycles(reset=True)
    out = h.run(xy, off, p, batched=True)
    enabled, cyc = h.phase_cycles(reset=True)
    assert h.status(out.status) == ref.status
    assert np.array_equal(out.npeaks.cpu().numpy(), ref.npeaks)
    assert np.array_equal(out.mask.cpu().numpy(), ref.mask)
    assert np.array_equal(out.nkept.cpu().numpy(), ref.nkept)
    pk = np.ascontiguousarray(out.peaks.cpu().numpy().astype(np.int16)).view(oracle.PEAK_DTYPE).reshape(ev.n_events, -1)
    for e in range(ev.n_events):  # the stored peak records, element by element
        s = min(int(ref.npeaks[e]), 512)
        assert np.array_equal(pk[e, :s], ref.peaks[e, :s]), e
    print(json.dumps({"enabled": enabled, "cycles": cyc, "lib": h.load()._name}))


if __name__ == "__main__":
    main()
