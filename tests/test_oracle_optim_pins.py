"""Pins of the fit loop's optimiser oracle (Adam with the paper's learning-rate
schedule, Sec. 5.1) against things other than itself: PyTorch's own Adam in
float64, the closed form of Adam under a constant gradient, the schedule's end
points, and finite differences through the log-scale / logit-intensity
parameterisation."""
import numpy as np
import pytest
import torch

from oracle import optim


def test_adam_matches_torch_adam_in_float64():
    rng = np.random.Generator(np.random.PCG64(1))
    theta0 = rng.standard_normal(37)
    p = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=3e-3, betas=(0.9, 0.999), eps=1e-15)
    theta, m, v = theta0.copy(), np.zeros(37), np.zeros(37)
    for t in range(1, 12):
        g = rng.standard_normal(37) * (1.0 + t)
        p.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        theta, m, v = optim.adam_update(theta, g, m, v, t, 3e-3)
        np.testing.assert_allclose(theta, p.detach().numpy(), rtol=1e-13, atol=1e-15)


def test_adam_constant_gradient_moves_lr_per_step():
    """With g constant, both bias-corrected moments equal g and g^2 exactly, so
    each step moves theta by lr * g / (|g| + eps) = lr sign(g)."""
    theta, m, v = np.array([0.0, 0.0, 1.0]), np.zeros(3), np.zeros(3)
    g = np.array([2.5, -0.25, 1e-3])
    for t in range(1, 40):
        theta, m, v = optim.adam_update(theta, g, m, v, t, 1e-2)
    np.testing.assert_allclose(theta, np.array([0.0, 0.0, 1.0]) - 39 * 1e-2 * np.sign(g), rtol=0, atol=1e-12)


def test_schedule_end_points():
    assert optim.lr_at(0.02, 1, 30000) == pytest.approx(0.02, rel=1e-15)
    assert optim.lr_at(0.02, 30001, 30000) == pytest.approx(0.002, rel=1e-12)
    assert optim.lr_at(0.02, 10 ** 6, 30000) == pytest.approx(0.002, rel=1e-12)
    assert optim.lr_at(0.02, 15001, 30000) == pytest.approx(0.02 * np.sqrt(0.1), rel=1e-12)  # geometric mid


def test_raw_parameter_gradients_by_finite_differences():
    """The state's update uses g_raw = dL/draw for L(params(raw)); check the
    chain g_log_s = g_s s and g_logit = g_a a (1 - a) against central
    differences of a smooth function of the activated parameters."""
    rng = np.random.Generator(np.random.PCG64(2))
    n = 4
    st = optim.FitState(rng.uniform(0, 9, (n, 3)), rng.uniform(0.5, 3, (n, 3)), rng.standard_normal((n, 4)),
                        rng.uniform(0.05, 0.95, n))
    W = {k: rng.standard_normal(st.raw[k].shape) for k in optim.GROUPS}

    def loss():
        mu, s, q, a = st.params()
        return float((W["mu"] * mu ** 2).sum() + (W["scale"] * s ** 2).sum() + (W["quat"] * q).sum()
                     + (W["alpha"] * a ** 3).sum())

    mu, s, q, a = st.params()
    grads = (2 * W["mu"] * mu, 2 * W["scale"] * s, W["quat"], 3 * W["alpha"] * a ** 2)
    g_raw = {"mu": grads[0], "scale": grads[1] * s, "quat": grads[2], "alpha": grads[3] * a * (1 - a)}
    for k in ("scale", "alpha"):
        flat = st.raw[k].reshape(-1)
        for i in range(flat.size):
            old = flat[i]
            flat[i] = old + 1e-6
            lp = loss()
            flat[i] = old - 1e-6
            lm = loss()
            flat[i] = old
            assert g_raw[k].reshape(-1)[i] == pytest.approx((lp - lm) / 2e-6, rel=1e-6, abs=1e-9)
    # and one state step moves the raw parameters by exactly the Adam step of g_raw
    raw0 = {k: v.copy() for k, v in st.raw.items()}
    st.step(grads, 1)
    for k in optim.GROUPS:
        lr = optim.PAPER_LR[k]
        exp_raw, _, _ = optim.adam_update(raw0[k], g_raw[k], np.zeros_like(raw0[k]), np.zeros_like(raw0[k]), 1, lr)
        np.testing.assert_allclose(st.raw[k], exp_raw, rtol=1e-15, atol=0)
