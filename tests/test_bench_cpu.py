"""Host-side helpers of the benchmark, on the CPU."""
import numpy as np

import bench


def test_fluence_l2_is_zero_for_the_sample_mean_and_scale_free():
    rng = np.random.default_rng(1)
    h1 = rng.poisson(50.0, (8, 8, 8)).astype(np.int64) << 20
    h2 = rng.poisson(50.0, (8, 8, 8)).astype(np.int64) << 20
    n_half = 1000
    # a GPU map equal to the sample's mean, at another packet count
    gpu = (h1 + h2) * 3
    r = bench.fluence_l2(gpu, 6 * n_half, (h1, h2), n_half)
    assert r["fluence_rel_l2"] < 1e-12
    # the sample's noise: half the difference of its halves, relative
    mean = (h1 + h2) / 2.0
    want = np.linalg.norm(h1 - h2.astype(float)) / 2.0 / np.linalg.norm(mean)
    assert abs(r["fluence_oracle_noise_rel_l2"] - want) < 1e-12
    # identical halves: no noise, no ratio
    assert bench.fluence_l2(gpu, 6 * n_half, (h1, h1), n_half)["fluence_l2_over_noise"] is None


def test_fluence_l2_matches_the_noise_for_a_consistent_estimate():
    # counts drawn around one expected map: a large-sample estimate differs
    # from the small sample by about the small sample's own noise
    rng = np.random.default_rng(2)
    lam = rng.uniform(5.0, 40.0, (10, 10, 10))
    n_half, n_gpu = 1, 400
    h1, h2 = rng.poisson(lam), rng.poisson(lam)
    gpu = rng.poisson(lam * n_gpu)
    r = bench.fluence_l2(gpu, n_gpu, (h1, h2), n_half)
    assert 0.7 < r["fluence_l2_over_noise"] < 1.4, r
