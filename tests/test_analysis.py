"""Measurement schedules: the log-spaced MSD grid against the paper's loop."""
import math

import numpy as np
import pytest

import oracle
from paper_2001_07089_gb300 import analysis


@pytest.mark.parametrize("n_md,t0,kmax", [(1000, 1.0, 60), (10000, 1.0, 60), (100000, 2.0, 40), (50, 1.0, 10)])
def test_log_grid_matches_oracle_loop(n_md, t0, kmax):
    assert analysis.log_time_grid(n_md, t0, kmax) == oracle.log_time_grid(n_md, t0, kmax)


def test_log_grid_shape_follows_eq_A():
    """Eq. (A): the k_max-th point lands on n_MD; points are distinct, increasing, and
    once they are far apart their ratios approach A."""
    n_md, kmax = 100000, 60
    g = analysis.log_time_grid(n_md, 1.0, kmax)
    A = n_md ** (1.0 / kmax)
    assert g[0] == 1 and g[-1] == n_md
    assert all(b > a for a, b in zip(g, g[1:]))
    assert len(g) <= kmax + 1
    tail = np.array(g[-10:], dtype=float)
    assert np.allclose(tail[1:] / tail[:-1], A, rtol=2e-3)
    # the first steps are consecutive integers while A*t grows by less than 1
    assert g[:5] == [1, 2, 3, 4, 5]
