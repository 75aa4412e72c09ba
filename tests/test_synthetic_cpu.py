"""The seeded input generators against the workloads they stand for: the forests' sizes and 2:1 balance, the batch
recipe's ranges, the log-normal coefficient's statistics, and seeding."""
import numpy as np
import pytest

import synthetic as syn
from oracle.octree_mg import check_forest


def _boxes(keys):
    """Integer boxes [lo, hi] of the leaves in units of the finest leaf's edge (R = 1 units scaled by R later)."""
    keys = np.asarray(keys, dtype=np.int64)
    top = int(keys[:, 0].max())
    size = 1 << (top - keys[:, 0])
    lo = keys[:, 1:] * size[:, None]
    return keys[:, 0], lo, lo + size[:, None]


def _max_level_jump_between_touching_leaves(keys):
    """Brute force over all leaf pairs whose closed boxes meet (face, edge or corner neighbours)."""
    lev, lo, hi = _boxes(keys)
    touch = np.all((lo[:, None, :] <= hi[None, :, :]) & (lo[None, :, :] <= hi[:, None, :]), axis=-1)
    np.fill_diagonal(touch, False)
    return int(np.abs(lev[:, None] - lev[None, :])[touch].max(initial=0))


@pytest.mark.parametrize("name,blocks,cells", [("sphere_2x32", (0, 56, 64), 3_932_160),
                                               ("sphere_4x32", (0, 448, 512), 31_457_280),
                                               ("uniform_8x64", (512,), 134_217_728)])
def test_workload_forests_have_the_stated_sizes(name, blocks, cells):
    R, n, keys = syn.workload_forest(name)
    check_forest(R, keys)
    counts = np.bincount([k[0] for k in keys], minlength=len(blocks))
    assert tuple(counts) == blocks
    assert len(keys) * n ** 3 == cells
    assert _max_level_jump_between_touching_leaves(keys) <= 1


def test_batch_recipe_ranges_and_balance():
    problems = syn.batch_problems(256, seed=0)
    assert len(problems) == 256
    ns = [n for n, _ in problems]
    assert set(ns) == {16, 32, 64, 128}
    depths = [max(k[0] for k in keys) for _, keys in problems]
    assert set(depths) == {0, 1, 2}
    for _, keys in problems:
        check_forest(1, keys)
        assert _max_level_jump_between_touching_leaves(keys) <= 1
    rows, pn = syn.batch_leaves(problems)
    assert rows.shape == (sum(len(k) for _, k in problems), 5) and list(pn) == ns
    assert np.all(np.diff(rows[:, 0]) >= 0)


def test_lognormal_k_has_the_stated_covariance():
    """log k is a zero-mean Gaussian field with covariance sigma^2 exp(-r^2 / (2 ell^2)) (sigma 1, ell 0.1):
    estimated over 24 seeds on a 32^3 grid (h = 1/32) at lags of 0 to 4 cells along each axis."""
    R, n = 1, 32
    keys = syn.uniform_leaves(R)
    ell, h = 0.1, 1.0 / n
    lags = range(5)
    est = np.zeros((3, len(lags)))
    means = []
    seeds = range(24)
    for s in seeds:
        g = np.log(syn.lognormal_k_rff(R, n, keys, seed=s).numpy().reshape(n, n, n))  # [z, y, x]
        means.append(g.mean())
        for a, ax in enumerate((2, 1, 0)):  # x, y, z
            for i, lag in enumerate(lags):
                p = np.take(g, range(0, n - lag), axis=ax)
                q = np.take(g, range(lag, n), axis=ax)
                est[a, i] += np.mean(p * q) / len(seeds)
    want = np.exp(-(np.asarray(list(lags)) * h) ** 2 / (2 * ell ** 2))
    assert abs(np.mean(means)) < 0.15
    np.testing.assert_allclose(est, np.broadcast_to(want, est.shape), atol=0.06)
    # the lag-4 value (r = 0.125) separates ell = 0.1 from ell = 0.05 (0.04) and 0.2 (0.82)
    assert 0.3 < est[:, 4].mean() < 0.65


def test_generators_are_seeded():
    R, n, keys = syn.workload_forest("sphere_2x8")
    a = syn.lognormal_k_rff(R, n, keys, seed=3)
    b = syn.lognormal_k_rff(R, n, keys, seed=3)
    c = syn.lognormal_k_rff(R, n, keys, seed=4)
    assert np.array_equal(a.numpy(), b.numpy()) and not np.array_equal(a.numpy(), c.numpy())
    f1 = syn.gaussian_bump_with_noise(R, n, keys, seed=5)
    f2 = syn.gaussian_bump_with_noise(R, n, keys, seed=5)
    assert np.array_equal(f1.numpy(), f2.numpy())
    assert syn.batch_problems(8, seed=1) == syn.batch_problems(8, seed=1)
