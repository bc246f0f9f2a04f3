"""GPU: the learned preconditioner sums (MLP trained by the library's kernels).

* gradients of one batch (tctl_mlp_grad, FP32 on the GPU) against the FP64
  oracle's chain-rule gradient (oracle/mlp.py, itself pinned by finite
  differences);
* training on fitter-generated sums lowers the dataset loss, and the GPU
  inference kernel reproduces the oracle's forward pass of the trained model;
* in the PCG: the learned sum is measured on the spectrum (delta) and used
  only below pre_delta_max, the solve matches the exact solution, and the
  network's nodes beat geometric nodes with the same number of terms on
  held-out problems (the gain over the method without the network).
"""
import math

import numpy as np
import pytest

from oracle import formats as F
from oracle import fullgrid as fg
from oracle import mlp
from oracle import operator as op
from paper_2006_09314_gb300.inputs import make_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # the marker deselects these on CPU hosts
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2006_09314_gb300 import tensorctl as T  # noqa: E402

R = 8


@pytest.fixture(scope="module")
def trained():
    X, Y, d = T.tctl_precond_dataset(R, 768, seed=11)
    model, loss = T.tctl_mlp_train(R, X, Y, steps=2500, batch=128, lr=3e-3, seed=5)
    return X, Y, d, model, loss


def test_mlp_gradients_match_oracle():
    O = 2 * R
    rng = np.random.default_rng(2)
    p = (rng.standard_normal(mlp.n_params(O)) * 0.2).astype(np.float32)
    X = rng.standard_normal((37, 4)).astype(np.float32)
    Tt = rng.standard_normal((37, O)).astype(np.float32)
    loss_g, g_g = T.tctl_mlp_grad(R, p, X, Tt)
    loss_o, g_o = mlp.loss_and_grad(p.astype(np.float64), X.astype(np.float64), Tt.astype(np.float64), O)
    assert loss_g == pytest.approx(loss_o, rel=1e-5)
    assert np.linalg.norm(g_g - g_o) <= 1e-5 * np.linalg.norm(g_o)
    assert np.max(np.abs(g_g - g_o)) <= 1e-5 * np.max(np.abs(g_o))


def test_training_lowers_loss_and_inference_matches_oracle(trained):
    X, Y, d, model, loss = trained
    assert np.all(np.isfinite(Y)) and np.all(d < 1.0)
    assert loss[1] < 0.2 * loss[0]
    O = 2 * R
    P = mlp.n_params(O)
    mu_in, sd_in = model[P:P + 4], model[P + 4:P + 8]
    mu_out, sd_out = model[P + 8:P + 8 + O], model[P + 8 + O:P + 8 + 2 * O]
    Xs = X[:50]
    Yo, _ = mlp.forward(model[:P].astype(np.float64), (Xs - mu_in) / sd_in, O)
    Yo = Yo * sd_out + mu_out
    Yg = T.tctl_mlp_forward(R, model, Xs)
    assert np.max(np.abs(Yg - Yo)) <= 1e-4 * (1.0 + np.max(np.abs(Yo)))


def _delta(theta, p, a, b, smin, smax, m=4000):
    s = np.exp(np.linspace(math.log(smin), math.log(smax), m))
    P = s * (np.exp(-np.outer(s, theta)) @ p)
    return float(np.max(np.abs(P * fg.F2(s, a, b) - 1.0)))


def test_network_nodes_beat_geometric_nodes(trained):
    """Held-out inputs: network nodes + NNLS weights vs geometric nodes + NNLS, same r."""
    from scipy.optimize import nnls
    _, _, _, model, _ = trained
    Xh, _, _ = T.tctl_precond_dataset(R, 24, seed=999)
    Yh = T.tctl_mlp_forward(R, model, Xh)
    wins, dl, dg = 0, [], []
    for x, y in zip(Xh.astype(np.float64), Yh.astype(np.float64)):
        a, b, smin, smax = x[0], 10 ** x[1], math.exp(x[2]), math.exp(x[3])
        s = np.exp(np.linspace(math.log(smin), math.log(smax), 300))
        fw = (s * fg.F2(s, a, b))[:, None]

        def weights(th):
            A = np.exp(-np.outer(s, th)) * fw
            cs = np.linalg.norm(A, axis=0)
            return nnls(A / cs, np.ones(s.size), maxiter=5000)[0] / cs
        th_l = np.exp(y[:R]) / smin
        th_g = np.exp(np.linspace(math.log(0.05 / smax), math.log(20 / smin), R))
        dl.append(_delta(th_l, weights(th_l), a, b, smin, smax))
        dg.append(_delta(th_g, weights(th_g), a, b, smin, smax))
        wins += dl[-1] < dg[-1]
    assert wins >= 18 and np.median(dl) < 0.5 * np.median(dg)


def test_learned_preconditioner_in_pcg(trained):
    _, _, _, model, _ = trained
    n, alpha, beta = 48, 0.5, 1e-2
    pr = make_problem(n, alpha, beta, 3, 42)
    lams, Vs = [], []
    for l in range(3):
        lam, V = op.eig(*op.assemble(pr.coeffs[l]))
        lams.append(lam)
        Vs.append(V)
    ustar = fg.solve_exact(F.cp_full(pr.yw, pr.yU), lams, Vs, alpha, beta)
    res = {}
    for src in (0, 2):
        o = T.tctl_default_opts(pre_src=src, pre_r=R, pre_model=model.ctypes.data, pre_delta_max=0.5)
        with T.Context(pr.coeffs, n, alpha, beta, 1e-6, opts=o) as ctx:
            x, st, _ = ctx.pcg_solve(T.CP.from_numpy(pr.yw, pr.yU))
            res[src] = (F.cp_full(*x.to_numpy()), st)
    u2, st2 = res[2]
    assert st2["pre_used"] == 2 and st2["pre_delta"] <= 0.5
    assert st2["pre_rank"] <= 3 * R < res[0][1]["pre_rank"]
    assert np.linalg.norm(u2 - ustar) <= 1e-6 * np.linalg.norm(ustar)
    # a bound the learned sum cannot meet sends the context back to the K-node sum
    o = T.tctl_default_opts(pre_src=2, pre_r=R, pre_model=model.ctypes.data, pre_delta_max=1e-9)
    with T.Context(pr.coeffs, n, alpha, beta, 1e-6, opts=o) as ctx:
        assert ctx.stats()["pre_used"] == 0


@pytest.fixture(scope="module")
def op_trained():
    r = 8
    X, Y, e = T.tctl_expsum_dataset(0, r, 768, seed=12)
    model, loss = T.tctl_mlp_train(r, X, Y, steps=2500, batch=128, lr=3e-3, seed=6)
    return r, model, loss


def test_learned_operator_head_judged_on_the_spectrum(op_trained):
    """Operator head (expsum_src 2): the network's r nodes of F2(s)/s, weights re-solved
    by NNLS. A loose judge accepts it, and the apply then follows the learned F2 to
    its measured error; the default judge (1e-7, which no r <= 16 sum of F2/s meets on
    these spectra) rejects it, the sinc quadrature takes over and the solve matches
    the exact solution to 1e-6."""
    r, model, loss = op_trained
    assert loss[1] < 0.2 * loss[0]
    n, alpha, beta = 40, 0.5, 1e-2   # s_max ~ 3e4: inside the training range of s_max
    pr = make_problem(n, alpha, beta, 3, 61)
    lams, Vs = [], []
    for l in range(3):
        lam, V = op.eig(*op.assemble(pr.coeffs[l]))
        lams.append(lam)
        Vs.append(V)
    X = F.cp_full(pr.yw, pr.yU)
    S = fg.spectral_sum(lams)
    exact = fg.apply_spectral(fg.F2(S, alpha, beta), X, Vs)
    o = T.tctl_default_opts(expsum_src=2, op_model=model.ctypes.data, op_r=r, op_judge=0.5)
    with T.Context(pr.coeffs, n, alpha, beta, 1e-6, opts=o) as ctx:
        st = ctx.stats()
        assert st["expsum_used"] == 2 and st["op_rank"] <= 3 * r
        e_l = st["op_learned_err"]
        assert 1e-7 < e_l < 0.5 and st["op_rel_err"] == e_l
        assert 0 < st["sinc24_err"] < 1e-2
        y = ctx.apply_op(T.CP.from_numpy(pr.yw, pr.yU))
    # the learned F2 is within e_l of F2 on the spectrum; the apply adds eps_trunc
    d = np.linalg.norm(F.cp_full(*y.to_numpy()) - exact) / np.linalg.norm(exact)
    assert d <= 1.5 * e_l + 2e-6
    o = T.tctl_default_opts(expsum_src=2, op_model=model.ctypes.data, op_r=r)
    with T.Context(pr.coeffs, n, alpha, beta, 1e-6, opts=o) as ctx:
        st = ctx.stats()
        assert st["expsum_used"] == 0 and st["op_learned_err"] > 1e-7
        assert st["op_rel_err"] <= 1e-8
        x, _, code = ctx.pcg_solve(T.CP.from_numpy(pr.yw, pr.yU))
    ustar = fg.solve_exact(X, lams, Vs, alpha, beta)
    assert code == 0
    assert np.linalg.norm(F.cp_full(*x.to_numpy()) - ustar) <= 1e-6 * np.linalg.norm(ustar)


def test_learned_operator_argument_errors(op_trained):
    r, model, _ = op_trained
    pr = make_problem(16, 0.5, 1e-2, 1, 1)
    for kw in (dict(expsum_src=2), dict(expsum_src=2, op_model=model.ctypes.data, op_r=40),
               dict(expsum_src=2, op_model=model.ctypes.data, op_judge=0.0), dict(expsum_src=3)):
        with pytest.raises(T.TctlError) as ei:
            T.tctl_setup(pr.coeffs, 16, 0.5, 1e-2, 1e-6, opts=T.tctl_default_opts(**kw))
        assert ei.value.code == -1
