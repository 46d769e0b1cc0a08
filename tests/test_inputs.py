"""The seeded input recipes: grids, masks, covariates and the serving stream have the sizes, shares
and distributions the workloads state, and are fixed by their seeds."""
import math

import numpy as np
import pytest

from paper_2012_13133_gb300 import inputs as I


def test_cell_centres_and_covariates():
    S1, S2 = I.cell_centres(4, 5)
    assert S1.shape == (4, 5)
    assert np.allclose(S1[:, 0], (np.arange(4) + 0.5) / 4) and np.allclose(S2[0], (np.arange(5) + 0.5) / 5)
    X = I.covariates(S1, S2)
    assert X.shape == (20, 3) and np.all(X[:, 0] == 1.0)
    assert np.array_equal(X[:, 1], S1.ravel()) and np.array_equal(X[:, 2], S2.ravel())


def test_uniform_mask_has_the_exact_missing_count_and_is_seeded():
    m = I.mask_uniform(30, 40, 0.37, 5)
    assert m.dtype == bool and m.shape == (30, 40)
    assert (~m).sum() == round(0.37 * 1200)
    assert np.array_equal(m, I.mask_uniform(30, 40, 0.37, 5))
    assert not np.array_equal(m, I.mask_uniform(30, 40, 0.37, 6))


def test_circle_mask_reaches_its_share_with_disc_shaped_gaps():
    n = 200
    m = I.mask_circles(n, n, 0.3, 4)
    miss = 1.0 - m.mean()
    # circles are added until the share is reached; the last may overshoot by one disc (r <= 0.15)
    assert 0.3 <= miss <= 0.3 + math.pi * 0.15 ** 2 + 1e-12
    # clustered: most missing cells have a missing 4-neighbour (a uniform mask at 30% gives ~76%)
    g = ~m
    nb = np.zeros_like(g)
    nb[1:] |= g[:-1]
    nb[:-1] |= g[1:]
    nb[:, 1:] |= g[:, :-1]
    nb[:, :-1] |= g[:, 1:]
    assert (g & nb).sum() >= 0.97 * g.sum()
    assert np.array_equal(m, I.mask_circles(n, n, 0.3, 4))


def test_mixed_mask_share():
    m = I.mask_mixed(128, 128, 0.6, 9)
    assert (~m).sum() >= round(0.6 * 128 * 128) - 1
    assert (~m).sum() <= round(0.6 * 128 * 128) + math.pi * 0.15 ** 2 * 128 * 128


@pytest.mark.parametrize("name,p", [("tiny32", 1024), ("grid1024", 524288), ("search512", 183501)])
def test_workload_masks_give_the_stated_observed_counts(name, p):
    w = I.WORKLOADS[name]
    assert int(I.make_mask(w).sum()) == p


def test_serving_stream_follows_its_recipe():
    reqs = I.serve_requests(2000, 4)
    assert len(reqs) == 2000
    t = np.array([r["arrival"] for r in reqs])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert gaps.mean() == pytest.approx(1.0, rel=0.1)                 # Exp(rate = 1)
    sides = np.array([r["n"] for r in reqs])
    assert sides.min() >= 128 and sides.max() <= 2048
    # log-uniform sides: the median is near sqrt(128 * 2048) = 512
    assert 400 <= np.median(sides) <= 650
    fm = np.array([r["frac_missing"] for r in reqs])
    assert fm.min() >= 0.1 and fm.max() <= 0.9
    assert {r["nu"] for r in reqs} == {0.5, 1.5}
    assert all(0.02 <= r["range"] <= 0.2 and 0.01 <= r["tau2"] <= 0.3 for r in reqs)
    share = np.mean([r["kind"] == "loglik" for r in reqs])
    assert 0.45 <= share <= 0.55
    assert reqs == I.serve_requests(2000, 4)


def test_data_noise_is_seeded_and_shaped():
    xi, eps = I.data_noise(8, 16, 10, 3)
    assert xi.shape == (2, 8, 16) and eps.shape == (10,)
    xi2, eps2 = I.data_noise(8, 16, 10, 3)
    assert np.array_equal(xi, xi2) and np.array_equal(eps, eps2)
    assert not np.array_equal(eps, I.normals(10, 3))       # the nugget noise is a separate stream


def test_variance_cells_are_a_seeded_sorted_choice_of_missing_cells():
    w = I.WORKLOADS["large4096"]
    n = 64
    mask = np.ones((n, n), bool)
    mask[10:30, 10:40] = False
    small = I.Workload("v", n, n, w.cov, "full", 0.0, 0, 0, extra={"n_var_cells": 100, "var_seed": 6})
    c1 = I.variance_cells(small, mask)
    c2 = I.variance_cells(small, mask)
    assert np.array_equal(c1, c2) and c1.dtype == np.int64 and c1.size == 100
    assert np.all(np.diff(c1) > 0) and not mask.ravel()[c1].any()
    # fewer missing cells than asked for: all of them
    mask[:] = True
    mask[0, :5] = False
    assert np.array_equal(I.variance_cells(small, mask), np.arange(5))
