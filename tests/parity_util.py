"""Helpers comparing the CUDA path's outputs with the CPU oracle (element by element)."""
import numpy as np

import oracle


def to_np(t):
    return t.detach().cpu().numpy()


def peaks_np(pk_t):
    """int16 [n_events, max_peaks, 4] -> oracle.PEAK_DTYPE [n_events, max_peaks]."""
    a = np.ascontiguousarray(to_np(pk_t).astype(np.int16))
    return a.view(oracle.PEAK_DTYPE).reshape(a.shape[0], a.shape[1])


def assert_event_outputs_equal(ref: "oracle.Result", npeaks, pk, mask, nkept, off, events=None, checksum=None,
                               max_peaks=None):
    """Exact comparison of per-event outputs. ``events`` selects which events of the GPU batch
    (by index) correspond to the oracle's events 0..len-1; ``off`` are the GPU batch offsets."""
    npeaks = to_np(npeaks)
    nkept = to_np(nkept)
    pk = peaks_np(pk)
    mask = to_np(mask)
    off = np.asarray(off)
    events = np.arange(len(npeaks)) if events is None else np.asarray(events)
    max_peaks = pk.shape[1] if max_peaks is None else max_peaks
    ref_off = np.zeros(len(events) + 1, np.int64)
    ref_off[1:] = np.cumsum(off[events + 1] - off[events])
    for i, e in enumerate(events):
        assert npeaks[e] == ref.npeaks[i], f"event {e}: npeaks {npeaks[e]} != {ref.npeaks[i]}"
        s = min(int(ref.npeaks[i]), max_peaks)
        if not np.array_equal(pk[e, :s], ref.peaks[i, :s]):
            bad = np.nonzero(pk[e, :s] != ref.peaks[i, :s])[0][:5]
            raise AssertionError(f"event {e}: peaks differ at {bad}: {pk[e, bad]} vs {ref.peaks[i, bad]}")
        assert nkept[e] == ref.nkept[i], f"event {e}: nkept {nkept[e]} != {ref.nkept[i]}"
        g = mask[off[e]:off[e + 1]]
        r = ref.mask[ref_off[i]:ref_off[i + 1]]
        if not np.array_equal(g, r):
            bad = np.nonzero(g != r)[0][:5]
            raise AssertionError(f"event {e}: mask differs at hits {bad}")
        if checksum is not None:
            c = to_np(checksum).view(np.uint64)
            assert c[e] == ref.checksum[i], f"event {e}: checksum {c[e]:#x} != {ref.checksum[i]:#x}"


def sub_batch(xy, off, events):
    """Hits of the given events as a batch of their own (for the oracle)."""
    events = np.asarray(events)
    parts = [xy[off[e]:off[e + 1]] for e in events]
    sub_off = np.zeros(len(events) + 1, np.int64)
    sub_off[1:] = np.cumsum([len(p) for p in parts])
    sub_xy = np.concatenate(parts) if parts else np.zeros((0, 2), np.int32)
    return sub_xy, sub_off
