"""CPU pins of the MLP oracle and of the r-term preconditioner fitter.

The oracle's analytic gradient is checked against central finite
differences of its own loss (a dropped term, wrong sign or transposed
weight in the chain rule fails this); the fitter's reported delta is
checked against the oracle's F2 on a denser grid, and its free nodes must
beat geometric nodes with NNLS weights at the same number of terms.
"""
import math

import numpy as np
import pytest
from scipy.optimize import nnls

from oracle import fullgrid as fg
from oracle import mlp


@pytest.mark.parametrize("O", [16, 24])
def test_oracle_gradient_matches_finite_differences(O):
    rng = np.random.default_rng(O)
    p = rng.standard_normal(mlp.n_params(O)) * 0.3
    X = rng.standard_normal((7, 4))
    T = rng.standard_normal((7, O))
    loss, g = mlp.loss_and_grad(p, X, T, O)
    assert loss == pytest.approx(mlp.loss_only(p, X, T, O), rel=1e-14)
    idx = rng.choice(p.size, 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (mlp.loss_only(p + e, X, T, O) - mlp.loss_only(p - e, X, T, O)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i]))


def test_oracle_forward_special_cases():
    O = 16
    p = np.zeros(mlp.n_params(O))
    W1, b1, W2, b2, W3, b3 = mlp.unpack(p, O)
    b3[:] = np.arange(O)
    Y, _ = mlp.forward(p, np.ones((3, 4)), O)
    assert np.array_equal(Y, np.tile(np.arange(O, dtype=float), (3, 1)))  # zero weights: biases


def _delta(theta, p, a, b, smin, smax, m=20000):
    s = np.exp(np.linspace(math.log(smin), math.log(smax), m))
    P = s * (np.exp(-np.outer(s, theta)) @ p)
    return float(np.max(np.abs(P * fg.F2(s, a, b) - 1.0)))


@pytest.mark.parametrize("a,b", [(0.25, 1e-4), (0.5, 1e-2), (0.75, 1.0)])
@pytest.mark.parametrize("r", [8, 12])
def test_precond_fit_delta_and_gain_over_geometric(a, b, r):
    from paper_2006_09314_gb300 import tensorctl as T
    smin, smax = 23.58, 6.57e7
    th, p, d = T.tctl_precond_fit(a, b, smin, smax, r)
    assert np.all(p > 0) and np.all(np.diff(th) >= 0) and th[0] > 0
    dd = _delta(th, p, a, b, smin, smax)
    assert dd <= 1.05 * d + 1e-12  # measured on 10x more points
    # geometric nodes over the same range with NNLS weights (the K-node default, at r)
    thg = np.exp(np.linspace(math.log(0.05 / smax), math.log(20 / smin), r))
    s = np.exp(np.linspace(math.log(smin), math.log(smax), 300))
    A = np.exp(-np.outer(s, thg)) * (s * fg.F2(s, a, b))[:, None]
    cs = np.linalg.norm(A, axis=0)
    pg = nnls(A / cs, np.ones(s.size), maxiter=5000)[0] / cs
    assert dd < _delta(thg, pg, a, b, smin, smax)
