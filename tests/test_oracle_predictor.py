"""Pins of the predictor reference (oracle/predictor.py) against facts that do
not come from itself: torch library ops for the network, central finite
differences for the gradient, and Adam's first step, which moves every
parameter by -lr * sign(g) (m_hat = g, v_hat = g^2 at step 1)."""
import numpy as np
import pytest

from oracle import predictor as P

DIMS = (7, 6, 4)  # in, hidden, out


def random_packed(seed, dims=DIMS):
    n_in, hid, n_out = dims
    off, total = P.layout(n_in, hid, n_out)
    g = np.random.default_rng(seed)
    p = g.standard_normal(total) * 0.5
    a, s = off["std"]
    p[a:a + s] = g.uniform(0.5, 2.0, s)
    a, s = off["scale"]
    p[a:a + s] = g.uniform(0.5, 2.0, s)
    return p


def test_network_against_torch():
    torch = pytest.importorskip("torch")
    n_in, hid, n_out = DIMS
    p = random_packed(1)
    v = P.unpack(p, *DIMS)
    x = np.random.default_rng(2).standard_normal((5, n_in))
    xt = (torch.tensor(x) - torch.tensor(v["mean"])) / torch.tensor(v["std"])
    F = torch.nn.functional
    h = F.silu(F.linear(xt, torch.tensor(v["W1"]), torch.tensor(v["b1"])))
    h = F.silu(F.linear(h, torch.tensor(v["W2"]), torch.tensor(v["b2"])))
    o = F.linear(h, torch.tensor(v["W3"]), torch.tensor(v["b3"])) * torch.tensor(v["scale"])
    assert np.allclose(P.forward(p, *DIMS, x), o.numpy(), rtol=1e-13, atol=1e-13)


def test_gradient_against_finite_differences():
    n_in, hid, n_out = DIMS
    p = random_packed(3)
    g = np.random.default_rng(4)
    x = g.standard_normal((9, n_in))
    t = g.standard_normal((9, n_out))
    loss, grad = P.loss_and_grad(p, *DIMS, x, t)
    begin = P.layout(*DIMS)[0]["W1"][0]
    for i in g.choice(grad.size, size=25, replace=False):
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[begin + i] += h
        pm[begin + i] -= h
        fd = (P.loss_and_grad(pp, *DIMS, x, t)[0] - P.loss_and_grad(pm, *DIMS, x, t)[0]) / (2 * h)
        assert abs(grad[i] - fd) <= 1e-7 * max(1.0, abs(fd)), (i, grad[i], fd)


def test_adam_first_step_moves_by_lr_times_sign():
    p = random_packed(5)
    g = np.random.default_rng(6)
    x = g.standard_normal((8, DIMS[0]))
    t = g.standard_normal((8, DIMS[2]))
    _, grad = P.loss_and_grad(p, *DIMS, x, t)
    n = grad.size
    p1, m, v, _ = P.train_step(p, np.zeros(n), np.zeros(n), *DIMS, x, t, lr=1e-3, step=1)
    begin = P.layout(*DIMS)[0]["W1"][0]
    big = np.abs(grad) > 1e-2  # eps / |g| <= 1e-6 there
    assert big.sum() > grad.size // 2
    assert np.allclose((p1 - p)[begin:][big], -1e-3 * np.sign(grad[big]), rtol=2e-6, atol=0)
    assert np.all(np.abs(p1 - p)[begin:] <= 1e-3 * (1 + 1e-12))  # Adam's first step is bounded by lr
    assert np.array_equal(p1[:begin], p[:begin])  # normalisation is not trained
