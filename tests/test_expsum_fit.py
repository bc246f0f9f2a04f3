"""Fitted exponential sums of F2(s)/s (expsum_src = 1), checked on the CPU.

The fitter runs on the host inside tctl_setup; tctl_expsum_fit exposes it
without a device. Its contract is the measured relative error of
F2(s) ~ s * sum_k w_k exp(-t_k s) (alpha < 1; sum + beta s at alpha = 1)
over the spectral interval (the same
measure as the sinc construction of Section 3.4), checked here against the
oracle's F2 on a grid 10x denser than the fitter's own check and on random
points, plus positivity of the weights (each term of g = F2/s is completely
monotone) and a term count below the sinc construction's.
"""
import math

import numpy as np
import pytest

from oracle import expsum as ox
from oracle import fullgrid as fg


def _fit(alpha, beta, smin, smax, tol):
    from paper_2006_09314_gb300 import tensorctl as T
    return T.tctl_expsum_fit(alpha, beta, smin, smax, tol)


# spectral intervals of the n = 256 and n = 2048 grids of the workload
@pytest.mark.parametrize("smin,smax", [(29.2, 1.3e6), (23.58, 6.57e7)])
@pytest.mark.parametrize("alpha", [0.25, 0.5, 0.75, 1.0])
@pytest.mark.parametrize("beta", [1e-4, 1e-2, 1.0])
def test_fitted_sum_meets_tolerance(alpha, beta, smin, smax):
    tol = 1e-8
    t, w, err = _fit(alpha, beta, smin, smax, tol)
    assert err <= tol
    assert np.all(w > 0) and np.all(t >= 0) and np.all(np.isfinite(t))
    rng = np.random.default_rng(7)
    s = np.concatenate([np.exp(np.linspace(math.log(smin), math.log(smax), 20000)),
                        np.exp(rng.uniform(math.log(smin), math.log(smax), 2000)), [smin, smax]])
    g = np.exp(-np.outer(s, t)) @ w
    approx = g + beta * s if alpha >= 1.0 else s * g
    exact = fg.F2(s, alpha, beta)
    # between the fitter's 2000 check points the error may rise a little
    assert np.max(np.abs(approx - exact) / exact) <= 1.5 * tol
    # Kronecker terms: 3 per node (s = sum of three eigenvalues) vs the sinc form
    rep = ox.F2_expsum(alpha, beta, smin, smax, tol)
    sinc_terms = len(rep["t1"]) + (3 if rep["exact_linear"] else 3 * len(rep["t2"]))
    fitted_terms = len(t) + 3 if alpha >= 1.0 else 3 * len(t)
    assert fitted_terms < sinc_terms


def test_fitted_sum_argument_errors():
    from paper_2006_09314_gb300 import tensorctl as T
    with pytest.raises(T.TctlError, match="E_ARG"):
        _fit(1.5, 1e-2, 20.0, 1e6, 1e-8)
    with pytest.raises(T.TctlError, match="E_ARG"):
        _fit(0.5, 1e-2, 1e6, 20.0, 1e-8)
    # a tolerance beyond FP64 reach is reported, not silently met
    with pytest.raises(T.TctlError, match="E_NUMERIC"):
        _fit(0.5, 1e-2, 20.0, 1e6, 1e-15)


@pytest.mark.parametrize("which", [0, 1])
def test_r_term_datasets_report_the_error_of_their_sums(which):
    """tctl_expsum_dataset: the error reported for every fitted r-term sum equals the
    error of that sum evaluated here from its (ln tau, ln q) against the oracle's F2
    (which 0: |s sum / F2 - 1|, the operator; which 1: |P F2 - 1|, P = s sum, the
    preconditioner), on the same 2000 log-spaced points; more terms fit better."""
    from paper_2006_09314_gb300 import tensorctl as T
    med = []
    for r in (6, 10):
        X, Y, e = T.tctl_expsum_dataset(which, r, 12, seed=77, threads=4)
        assert np.all(np.isfinite(Y)) and np.all(e > 0)
        for x, y, ek in zip(X.astype(np.float64), Y.astype(np.float64), e):
            a, b, smin, smax = x[0], 10 ** x[1], math.exp(x[2]), math.exp(x[3])
            assert 0.1 <= a <= 0.9 and 1e-4 <= b <= 1.0
            s = np.exp(np.linspace(math.log(smin), math.log(smax), 2000))
            f2 = fg.F2(s, a, b)
            target = f2 / s if which == 0 else 1.0 / (s * f2)
            t0 = f2[0] / s[0] if which == 0 else 1.0 / (s[0] * f2[0])
            tau, q = np.exp(y[:r]), np.exp(y[r:])
            assert np.all(np.diff(tau) >= 0)                     # ascending nodes
            v = (q[None, :] * np.exp(-np.outer(s / smin, tau))).sum(1) * t0
            err = np.max(np.abs(v / target - 1.0))
            # targets are stored in float32: ln tau, ln q to ~6e-8 relative
            assert err == pytest.approx(ek, rel=2e-3, abs=2e-5)
        med.append(np.median(e))
    assert med[1] < med[0]


def test_dataset_argument_errors():
    from paper_2006_09314_gb300 import tensorctl as T
    for which, r, n in [(2, 8, 4), (0, 1, 4), (1, 8, 0)]:
        with pytest.raises(T.TctlError) as ei:
            T.tctl_expsum_dataset(which, r, n)
        assert ei.value.code == -1
