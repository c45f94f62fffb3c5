"""The seeded input generator (CPU): the log-normal permeability field has the
stated distribution, correlation and reproducibility, and the workload
recipes have the stated sizes."""
import numpy as np
import pytest

from paper_2108_13229_gb300 import inputs as I


def test_reproducible_and_seeded():
    a = I.lognormal_K(64, -4.0, 1.0, 16.0, seed=3)
    b = I.lognormal_K(64, -4.0, 1.0, 16.0, seed=3)
    c = I.lognormal_K(64, -4.0, 1.0, 16.0, seed=4)
    assert a.shape == (64, 64) and np.all(a > 0) and np.all(np.isfinite(a))
    assert np.array_equal(a, b)
    assert not np.allclose(a, c)


@pytest.mark.parametrize("n", [32, 128, 1024])
def test_embedding_needs_no_clipping(n):
    # the exponential covariance on the padded torus is positive definite at
    # these sizes: no eigenvalue is clipped, so the field is exact in law
    _, info = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=0, return_info=True)
    assert info["clipped_fraction"] == 0.0
    assert info["embed"] >= max(2 * n, n + 128) and info["embed"] & (info["embed"] - 1) == 0


def test_lognormal_covariance():
    # 400 fields of 32 x 32 cells, ln K ~ N(-4, 1.5^2) with correlation length
    # 4 cells: with the known mean, the ensemble covariance of ln K at axis and
    # diagonal lags is sigma^2 exp(-r / ell), the same in x and y (isotropic,
    # not separable); a Gaussian kernel, a missing square on sigma or a lag in
    # the wrong unit fails it
    n, ell, sig = 32, 4.0, 1.5
    g = (np.stack([np.log(I.lognormal_K(n, -4.0, sig, ell, seed=s)) for s in range(400)]) + 4.0) / sig
    assert abs(g.mean()) < 0.05
    for dy, dx in [(0, 0), (0, 4), (4, 0), (0, 8), (8, 0), (0, 12), (12, 0), (3, 4), (6, 8)]:
        c = float((g[:, : n - dy, : n - dx] * g[:, dy:, dx:]).mean())
        assert abs(c - np.exp(-np.hypot(dx, dy) / ell)) < 0.04, (dy, dx, c)


def test_lognormal_statistics_at_workload_scale():
    # ln K ~ N(-4, 1) with correlation length 16 cells on 128 x 128 cells: the
    # ensemble mean and variance, and correlation falling with the lag
    n, ell = 128, 16.0
    g = np.stack([np.log(I.lognormal_K(n, -4.0, 1.0, ell, seed=s)) for s in range(8)]) + 4.0
    assert abs(g.mean()) < 0.25
    var = float((g * g).mean())
    assert 0.7 < var < 1.3
    corr = [float((g[:, :, : n - k] * g[:, :, k:]).mean()) / var for k in (16, 48)]
    assert abs(corr[0] - np.exp(-1.0)) < 0.12 and corr[0] > corr[1] and abs(corr[1]) < 0.2


def test_sigma_and_mean_scale_the_field():
    # the same seed draws the same standard field: ln K = mean + sigma * g
    g1 = np.log(I.lognormal_K(48, 0.0, 1.0, 8.0, seed=11))
    g2 = np.log(I.lognormal_K(48, -3.0, 2.0, 8.0, seed=11))
    assert np.allclose(g2, -3.0 + 2.0 * g1, rtol=0, atol=1e-12)


def test_workload_recipes():
    wl = I.lognormal_at_scale(1024)
    assert (wl.n, wl.mu, wl.alpha, wl.dt) == (1024, 1e-3, 1.0, 0.05) and wl.dof == 4196352
    assert I.mms_small().dof == 4160
    batch = I.batch_instances(256, seed=0)
    assert len(batch) == 256 and {w.n for w in batch} <= {64, 128, 256, 512}
    assert all(0.5 <= w.K_sigma <= 2.0 and 0.1 <= w.alpha <= 10.0 for w in batch)
    reqs = I.serving_requests(50, 10.0, seed=0)
    t = [ta for ta, _ in reqs]
    assert len(reqs) == 50 and t == sorted(t)
    assert all(32 <= w.n <= 1024 and 5 <= w.steps <= 50 for _, w in reqs)


def test_serving_mix_is_log_uniform():
    # 4000 requests at 50 req/s: sizes m * 2^k (m in 4..8) spanning 32..1024
    # log-uniformly (a fifth of the draws at 512 or above, median near the
    # geometric mean 181), lengths 5..50 steps, exponential inter-arrival
    # times with mean 1 / rate
    reqs = I.serving_requests(4000, 50.0, seed=1)
    n = np.array([w.n for _, w in reqs])
    assert n.min() == 32 and n.max() == 1024
    for v in np.unique(n).tolist():
        assert any(v % 2**k == 0 and 4 <= v // 2**k <= 8 for k in range(11)), v
    assert 0.15 < np.mean(n >= 512) < 0.25
    assert 128 <= np.median(n) <= 256
    steps = np.array([w.steps for _, w in reqs])
    assert steps.min() == 5 and steps.max() == 50
    t = np.array([ta for ta, _ in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0) and abs(gaps.mean() * 50.0 - 1.0) < 0.05
