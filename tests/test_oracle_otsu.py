"""Pins the oracle's Otsu objective and histogram (thresholding application,
Sec. 5.2) to textbook identities and exhaustive search."""
import itertools

import numpy as np
import pytest

from paper_2510_14982_gb300 import inputs


def test_histogram_matches_bincount(orc):
    px = inputs.gmm_image(3, 50_000)
    np.testing.assert_array_equal(orc.histogram_u8(px), np.bincount(px, minlength=256))


@pytest.mark.parametrize("T", [1, 2, 4, 8])
def test_between_class_variance_is_total_minus_within(orc, T):
    """Law of total variance on the pixels themselves: sigma_B^2 = sigma^2 - sum_c w_c sigma_c^2."""
    px = inputs.gmm_image(T, 40_000).astype(np.float64)
    hist = np.bincount(px.astype(np.int64), minlength=256)
    rng = np.random.default_rng(T)
    for _ in range(5):
        t = np.sort(rng.integers(0, 256, T))
        labels = np.searchsorted(t, px, side="left")   # class c holds (t_{c-1}, t_c]
        within = 0.0
        for c in np.unique(labels):
            v = px[labels == c]
            within += v.size / px.size * v.var()
        want = px.var() - within
        got = orc.otsu_sigma_b2(hist, t)
        assert got == pytest.approx(want, rel=1e-9, abs=1e-9)


def test_objective_uses_floor_of_positions_and_sorts(orc):
    px = inputs.gmm_image(1, 20_000)
    hist = np.bincount(px, minlength=256)
    p = orc.OracleProblem.from_spec(inputs.otsu_problem(hist, 3))
    f1 = orc.objective(p, np.array([100.7, 20.2, 180.999]))[0]
    f2 = -orc.otsu_sigma_b2(hist, np.array([20, 100, 180]))
    assert f1 == f2
    # clamped at the range ends
    f3 = orc.objective(p, np.array([-5.0, 300.0, 255.0]))[0]
    assert f3 == -orc.otsu_sigma_b2(hist, np.array([0, 255, 255]))


def _bimodal_hist(seed, n=30_000, bins=256):
    rng = np.random.default_rng(seed)
    a = rng.normal(0.3 * bins, 0.06 * bins, n // 2)
    b = rng.normal(0.7 * bins, 0.08 * bins, n - n // 2)
    v = np.clip(np.rint(np.concatenate([a, b])), 0, bins - 1).astype(np.int64)
    h = np.zeros(256, np.int64)
    h[:bins] = np.bincount(v, minlength=bins)
    return h


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_apo_reaches_exhaustive_optimum_one_threshold(orc, seed):
    hist = _bimodal_hist(seed)
    best = max(orc.otsu_sigma_b2(hist, np.array([t])) for t in range(256))
    p = orc.OracleProblem.from_spec(inputs.otsu_problem(hist, 1))
    _, bf, _ = orc.apo_run(p, orc.params(ps=100, pf_max=0.1, max_iter=50, seed=seed))
    assert -bf == best


def test_apo_reaches_exhaustive_optimum_two_thresholds(orc):
    hist = _bimodal_hist(5)
    best = max(orc.otsu_sigma_b2(hist, np.array([a, b]))
               for a in range(256) for b in range(a, 256))
    p = orc.OracleProblem.from_spec(inputs.otsu_problem(hist, 2))
    _, bf, _ = orc.apo_run(p, orc.params(ps=100, pf_max=0.1, max_iter=200, seed=1))
    assert -bf == pytest.approx(best, rel=1e-12)


@pytest.mark.parametrize("T", [3, 4])
def test_apo_reaches_exhaustive_optimum_toy_16_bins(orc, T):
    rng = np.random.default_rng(T)
    hist = np.zeros(256, np.int64)
    hist[:16] = rng.integers(0, 200, 16)
    best = max(orc.otsu_sigma_b2(hist, np.array(c))
               for c in itertools.combinations_with_replacement(range(16), T))
    spec = inputs.otsu_problem(hist, T)
    spec.ub = np.full(T, 15.999)
    p = orc.OracleProblem.from_spec(spec)
    _, bf, _ = orc.apo_run(p, orc.params(ps=100, pf_max=0.1, max_iter=300, seed=2))
    assert -bf == pytest.approx(best, rel=1e-12)
