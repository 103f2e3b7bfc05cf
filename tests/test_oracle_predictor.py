"""Pins of the predictor reference (oracle/predictor.py) against facts that do
not come from itself: torch library ops for the network, central finite
differences for the gradient, Adam's first step, which moves every
parameter by -lr * sign(g) (m_hat = g, v_hat = g^2 at step 1), and Adam's second
step against its closed form from the two gradients."""
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


def test_adam_second_step_closed_form():
    """Unrolling Kingma & Ba's moments over two steps from m = v = 0:
        m_2 = (1 - b1)(b1 g_1 + g_2),  v_2 = (1 - b2)(b2 g_1^2 + g_2^2),
    and with the bias corrections 1 - b^2 = (1 - b)(1 + b),
        m_hat = (b1 g_1 + g_2) / (1 + b1),  v_hat = (b2 g_1^2 + g_2^2) / (1 + b2),
    so p_2 = p_1 - lr m_hat / (sqrt(v_hat) + eps).  Swapping b1 and b2, or a bias
    correction with the wrong power, moves p_2 off this value."""
    b1, b2, eps, lr = 0.9, 0.999, 1e-8, 1e-3
    p0 = random_packed(7)
    g = np.random.default_rng(8)
    x = g.standard_normal((8, DIMS[0]))
    t = g.standard_normal((8, DIMS[2]))
    n = P.loss_and_grad(p0, *DIMS, x, t)[1].size
    begin = P.layout(*DIMS)[0]["W1"][0]
    _, g1 = P.loss_and_grad(p0, *DIMS, x, t)
    p1, m1, v1, _ = P.train_step(p0, np.zeros(n), np.zeros(n), *DIMS, x, t, lr=lr, step=1)
    _, g2 = P.loss_and_grad(p1, *DIMS, x, t)
    p2, m2, v2, _ = P.train_step(p1, m1, v1, *DIMS, x, t, lr=lr, step=2)
    assert np.allclose(m2, (1 - b1) * (b1 * g1 + g2), rtol=1e-13, atol=1e-300)
    assert np.allclose(v2, (1 - b2) * (b2 * g1 ** 2 + g2 ** 2), rtol=1e-13, atol=1e-300)
    m_hat = (b1 * g1 + g2) / (1 + b1)
    v_hat = (b2 * g1 ** 2 + g2 ** 2) / (1 + b2)
    want = p1[begin:] - lr * m_hat / (np.sqrt(v_hat) + eps)
    assert np.allclose(p2[begin:], want, rtol=1e-12, atol=1e-15)
    assert np.array_equal(p2[:begin], p0[:begin])
    # the step differs from Adam's first-step form: both gradients enter
    assert not np.allclose(p2[begin:] - p1[begin:], -lr * np.sign(g2), rtol=1e-3, atol=0)
