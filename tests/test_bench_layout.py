"""Host logic of the benchmark's part layout: parts grouped into surfel-count bands, each
band contiguous (so the end-to-end step can copy a band's data in one piece), and the
seeded part index -> position map that keeps the served trace and the batched-vs-plain
subset independent of the layout."""
import numpy as np

import bench


def _check(ns, thresholds):
    orig, band = bench.band_layout(ns, thresholds)
    P = len(ns)
    assert sorted(orig.tolist()) == list(range(P))          # a permutation
    assert np.all(np.diff(band) >= 0)                        # bands contiguous, in order
    bounds = [float("inf")] + list(thresholds)
    for i, s in enumerate(orig):
        j = band[i]
        if j < len(thresholds):
            assert bounds[j + 1] <= ns[s] < bounds[j]
        else:
            assert all(not (bounds[k + 1] <= ns[s] < bounds[k]) for k in range(len(thresholds)))
    for j in np.unique(band):                                # seeded order within a band
        assert np.all(np.diff(orig[band == j]) > 0)
    at = bench.seeded_positions(orig)
    assert np.array_equal(at[orig], np.arange(P))
    assert np.array_equal(np.asarray(ns)[orig][at], np.asarray(ns))
    return orig, band


def test_band_layout_random_batches():
    g = np.random.default_rng(5)
    for _ in range(20):
        P = int(g.integers(1, 400))
        ns = np.exp(g.normal(np.log(20000), 1.2, P)).astype(np.int64).clip(1000, 500000)
        _check(ns, [350000, 150000])
        _check(ns, [100000])


def test_band_layout_edges():
    # values on the thresholds go to the band whose lower bound they meet
    ns = np.array([150000, 149999, 350000, 349999, 500000, 1])
    orig, band = _check(ns, [350000, 150000])
    assert orig.tolist() == [2, 4, 0, 3, 1, 5]
    assert band.tolist() == [0, 0, 1, 1, 2, 2]
    # no thresholds: one band, identity layout
    orig, band = _check(ns, [])
    assert orig.tolist() == list(range(6)) and band.tolist() == [0] * 6
    # an empty band keeps the others contiguous
    orig, band = _check(np.array([10, 20, 400000]), [350000, 150000])
    assert band.tolist() == [0, 2, 2]
