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


def test_paired_block_stats_accepts_equal_expectations_and_rejects_a_local_bias():
    # K batches of n blocks: both sides noisy around one expected map
    rng = np.random.default_rng(3)
    K, n = 40, 800
    lam = rng.uniform(200.0, 2000.0, n)
    A = rng.poisson(lam, (K, n)).astype(float)
    B = rng.poisson(lam, (K, n)).astype(float)
    r = bench.paired_block_stats(A, B)
    assert r["blocks"] == n and r["pass"], r
    assert abs(r["chi2_dof"] - 1.0) < r["chi2_band"]
    # a 6 % bias in 1 % of the blocks (a few wrong voxels near a surface):
    # an L2 norm over the map would not see it, the block z-scores do
    Bb = B.copy()
    Bb[:, :8] *= 1.06
    rb = bench.paired_block_stats(A, Bb)
    assert not rb["pass"], rb
    # blocks that are empty in some batch are left out
    A2 = A.copy()
    A2[5, :10] = 0
    assert bench.paired_block_stats(A2, B)["blocks"] == n - 10


def test_paired_block_stats_correlated_blocks():
    # every block shares one batch-level fluctuation (packets that cross many
    # blocks): the effective block count is small and the chi2 band widens
    rng = np.random.default_rng(4)
    K, n = 40, 500
    common = rng.normal(0.0, 1.0, (K, 1))
    A = 1000.0 + 10.0 * (common + 0.3 * rng.normal(0.0, 1.0, (K, n)))
    B = 1000.0 + 10.0 * (0.3 * rng.normal(0.0, 1.0, (K, n)))
    r = bench.paired_block_stats(A, B)
    assert r["n_eff"] < 0.2 * n, r
    assert r["pass"], r


def test_paired_z():
    rng = np.random.default_rng(5)
    x = rng.normal(1.0, 1.0, 10000)
    y = x + rng.normal(0.0, 0.01, 10000)
    assert abs(bench.paired_z(x, y)) < 4
    assert bench.paired_z(x, y - 0.001) > 5


def test_unpaired_block_stats():
    # an independent small sample (few batches, few packets) against a large
    # one: Welch degrees of freedom; equal expectations pass, a local bias fails
    rng = np.random.default_rng(6)
    n = 300
    lam = rng.uniform(50.0, 500.0, n)
    A = rng.poisson(lam, (20, n)).astype(float)
    B = rng.poisson(lam * 100, (10, n)).astype(float) / 100
    r = bench.block_stats(A, B, paired=False)
    assert r["pass"], r
    Bb = B.copy()
    Bb[:, :6] *= 1.25
    assert not bench.block_stats(A, Bb, paired=False)["pass"]
