"""Host logic of the refinement (no GPU): the library's marking and splitting
(pff_mark_axes, the step pff_refine_axes runs after its device reductions)
against the oracle's mark_intervals + split_intervals, bit for bit, on random
and hand-made slab data (ties with the threshold, zero sums, theta > 1, intervals
exactly h_band long, minima exactly at phi_band), and its argument checks."""
import numpy as np
import pytest

from oracle import adapt

pff = pytest.importorskip("paper_1806_09924_gb300")


def _oracle(coords, S, P, theta, h_band, phi_band):
    return adapt.split_intervals(coords, adapt.mark_intervals(coords, S, P, theta, h_band, phi_band))


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("seed", range(6))
def test_random_slab_data_matches_oracle(dim, seed):
    rng = np.random.default_rng(seed)
    coords = [np.cumsum(np.concatenate([[-1.0], rng.uniform(0.01, 0.3, rng.integers(1, 40))]))
              for _ in range(dim)]
    S = [rng.exponential(size=len(c) - 1) * (rng.random(len(c) - 1) < 0.8) for c in coords]
    P = [rng.random(len(c) - 1) for c in coords]
    for theta, h_band, phi_band in ((0.3, 0.1, 0.5), (0.0, 0.0, 0.0), (2.0, 0.05, 0.9), (1.0, 1.0, 1.0)):
        got = pff.mark_axes(coords, S, P, theta, h_band, phi_band)
        ref = _oracle(coords, S, P, theta, h_band, phi_band)
        for g, r in zip(got, ref):
            np.testing.assert_array_equal(g, r)


def test_hand_made_boundaries_match_oracle():
    x = np.array([0.0, 1.0, 1.5, 3.0, 3.125, 3.25])
    y = np.array([0.0, 0.5, 1.0])
    S = [np.array([0.0, 0.25, 1.0, 0.25, 0.0]), np.array([0.0, 0.0])]
    P = [np.array([1.0, 0.5, 1.0, 0.25, 0.0]), np.array([0.5, 0.49])]
    for theta in (0.25, 0.26, 1.0, 1.5):
        for h_band in (0.125, 0.0625, 0.5):
            got = pff.mark_axes([x, y], S, P, theta, h_band, 0.5)
            ref = _oracle([x, y], S, P, theta, h_band, 0.5)
            for g, r in zip(got, ref):
                np.testing.assert_array_equal(g, r)
    # theta = 0.25: the slabs with S = 0.25 sit exactly on the threshold and split
    got = pff.mark_axes([x, y], S, P, 0.25, 0.5, 0.0)
    np.testing.assert_array_equal(got[0], [0.0, 1.0, 1.25, 1.5, 2.25, 3.0, 3.0625, 3.125, 3.25])
    np.testing.assert_array_equal(got[1], y)   # all-zero sums, no slab below phi_band = 0


def test_argument_checks():
    x = np.array([0.0, 1.0, 2.0])
    with pytest.raises(pff.PffError):
        pff.mark_axes([x, np.array([0.0, 1.0, 0.5])], [np.ones(2), np.ones(2)], [np.ones(2)] * 2, 0.3, 0.1, 0.5)
    with pytest.raises(pff.PffError):
        pff.mark_axes([x, x], [np.ones(2)] * 2, [np.ones(2)] * 2, -0.1, 0.1, 0.5)
    with pytest.raises(pff.PffError):
        pff.mark_axes([x, x], [np.ones(2)] * 2, [np.ones(2)] * 2, 0.3, float("nan"), 0.5)
    with pytest.raises(pff.PffError):
        pff.mark_axes([x], [np.ones(2)], [np.ones(2)], 0.3, 0.1, 0.5)
