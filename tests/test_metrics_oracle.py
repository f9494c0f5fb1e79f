"""Pins of the oracle's flow metrics (oracle/metrics.py): the similarity index of Sec. 3.4 on
cases whose value follows from its definition, and the time mean."""
import numpy as np

from oracle import metrics as M


def _field(seed, shape=(4, 5, 6)):
    return np.random.default_rng(seed).normal(size=(3,) + shape)


def test_identical_fields_score_one():
    u = _field(0)
    assert abs(M.similarity_index(u, u, np.ones(u.shape[1:])) - 1.0) < 1e-15


def test_scaled_field_scores_one_and_reversed_scores_zero():
    u = _field(1)
    m = np.ones(u.shape[1:])
    assert abs(M.similarity_index(u, 3.5 * u, m) - 1.0) < 1e-14   # magnitudes are normalised by their maxima
    assert abs(M.similarity_index(u, -u, m)) < 1e-15               # cos = -1 everywhere


def test_two_point_hand_value():
    # point 1: u_a = (1,0,0), u_b = (0,2,0): cos 0, |u_a|/max = 1, |u_b|/max = 1 -> 1/2
    # point 2: u_a = (0.5,0,0), u_b = (0,2,0)... |u_a|/max = .5, |u_b|/max = 1, cos 0 -> 1/2 * 1/2
    ua = np.array([[1.0, 0.5], [0.0, 0.0], [0.0, 0.0]])
    ub = np.array([[0.0, 0.0], [2.0, 2.0], [0.0, 0.0]])
    assert abs(M.similarity_index(ua, ub, np.ones(2)) - (0.5 + 0.25) / 2) < 1e-15


def test_mask_selects_points_and_maxima():
    u = _field(2)
    v = u.copy()
    m = np.zeros(u.shape[1:])
    m[1, 2, :] = 1
    v[:, 0] = -7.0  # outside the mask: must not change the score or the maxima
    assert abs(M.similarity_index(u, v, m) - 1.0) < 1e-14


def test_zero_vector_point():
    ua = np.array([[1.0, 0.0], [0.0, 0.0], [0.0, 0.0]])
    ub = np.array([[1.0, 1.0], [0.0, 0.0], [0.0, 0.0]])
    # point 2: u_a = 0 -> cos 0, magnitudes 0 vs 1 -> 1/2 * 0 = 0; point 1 scores 1
    assert abs(M.similarity_index(ua, ub, np.ones(2)) - 0.5) < 1e-15


def test_time_mean():
    xs = [np.full((2, 3), float(k)) for k in range(5)]
    assert np.array_equal(M.time_mean(xs), np.full((2, 3), 2.0))
