"""hough_run_batched_static: the batched path for callers that cannot allocate device memory.

Such callers (a trigger process that only owns the input and output buffers its readout layer
mapped, or a real-time loop that may not call cudaMalloc after start-up) get the scratch from a
fixed array inside the library. This file is collected last on purpose; it checks, through the
C ABI, that two calls in a row give exactly what hough_run_batched gives, and that a batch too
large for the built-in array is refused.
"""
import numpy as np
import pytest

import gen
from parity_util import peaks_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_04067_gb300 as hough
    hough.load()
    return hough


def same(h, a, b):
    assert h.status(a.status) == h.status(b.status)  # 0, or the peak-overflow flag in both
    assert torch.equal(a.npeaks, b.npeaks) and torch.equal(a.nkept, b.nkept) and torch.equal(a.mask, b.mask)
    assert torch.equal(a.checksum, b.checksum)
    pa, pb = peaks_np(a.peaks), peaks_np(b.peaks)
    for e in range(len(pa)):
        n = min(int(a.npeaks[e]), pa.shape[1])
        assert np.array_equal(pa[e, :n], pb[e, :n]), e


@pytest.mark.parametrize("name,n,tiles,max_peaks,iterative",
                         [("plain_paper", 300, 0, 2048, False), ("plain_paper", 60, 2, 512, False),
                          ("plain_small", 100, 0, 1024, False), ("plain_paper", 300, 0, 2048, True)])
def test_static_scratch_matches_workspace_path_twice(h, name, n, tiles, max_peaks, iterative):
    cfg = gen.CONFIGS[name]
    ev = gen.generate(cfg, n)
    xy, off = torch.from_numpy(ev.xy).cuda(), torch.from_numpy(ev.off).cuda()
    kw = dict(peak_mode=1, rel_num=1, rel_den=2, nms_radius=3) if iterative else {}
    p = h.params(cfg.n_theta, cfg.n_rho, cfg.threshold, cfg.keep_halfwidth, max_peaks, theta_tiles=tiles, **kw)
    assert h.workspace_size(p, ev.n_events) <= 32 * 1024 * 1024
    ref = h.run(xy, off, p, checksum=True, batched=True)
    for _ in range(2):  # the array keeps the previous call's contents; results must not depend on them
        out = h.alloc_outputs(ev.n_hits, ev.n_events, p, checksum=True)
        out.mask.fill_(9)
        h.run_static(xy, off, p, out)
        same(h, ref, out)


def test_static_scratch_rejects_oversized_batch(h):
    cfg = gen.CONFIGS["plain_paper"]
    ev = gen.generate(cfg, 8)
    p = h.params(256, 256, 16, 1, 65536, theta_tiles=8)  # tile peak slots: 8 events x 8 x 65536 x 8 B > 32 MiB
    assert h.workspace_size(p, ev.n_events) > 32 * 1024 * 1024
    out = h.alloc_outputs(ev.n_hits, ev.n_events, p)
    with pytest.raises(h.HoughError) as ei:
        h.run_static(torch.from_numpy(ev.xy).cuda(), torch.from_numpy(ev.off).cuda(), p, out)
    assert ei.value.code == h.EWORKSPACE
