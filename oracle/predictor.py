"""FP64 reference of the learned Newton predictor (TEST INFRASTRUCTURE ONLY).

Plain numpy: the network and one Adam training step written from their
definitions, for checking the CUDA inference and training kernels.

Packed vector (in features, H hidden, out outputs):
    mean[in] std[in] scale[out] W1[H][in] b1[H] W2[H][H] b2[H] W3[out][H] b3[out]
network(x) = W3 silu(W2 silu(W1 xn + b1) + b2) + b3,  xn = (x - mean) / std,
prediction = network(x) * scale, silu(z) = z / (1 + exp(-z)).
Loss of a batch: mean over samples and outputs of (network(x) - t / scale)^2.
Adam (Kingma & Ba 2015): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
p -= lr (m / (1 - b1^k)) / (sqrt(v / (1 - b2^k)) + eps), b1 = 0.9, b2 = 0.999,
eps = 1e-8, k = step >= 1.
"""
import numpy as np


def layout(n_in, hid, n_out):
    sizes = [("mean", n_in), ("std", n_in), ("scale", n_out), ("W1", hid * n_in), ("b1", hid),
             ("W2", hid * hid), ("b2", hid), ("W3", n_out * hid), ("b3", n_out)]
    off, pos = {}, 0
    for name, size in sizes:
        off[name] = (pos, size)
        pos += size
    return off, pos


def unpack(packed, n_in, hid, n_out):
    off, _ = layout(n_in, hid, n_out)
    p = np.asarray(packed, dtype=np.float64)
    v = {k: p[a:a + s] for k, (a, s) in off.items()}
    v["W1"] = v["W1"].reshape(hid, n_in)
    v["W2"] = v["W2"].reshape(hid, hid)
    v["W3"] = v["W3"].reshape(n_out, hid)
    return v


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_d(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s + z * s * (1.0 - s)


def network(v, x):
    """Returns (output in normalised units, cache for backprop)."""
    xn = (np.asarray(x, dtype=np.float64) - v["mean"]) / v["std"]
    z1 = xn @ v["W1"].T + v["b1"]
    h1 = silu(z1)
    z2 = h1 @ v["W2"].T + v["b2"]
    h2 = silu(z2)
    o = h2 @ v["W3"].T + v["b3"]
    return o, (xn, z1, h1, z2, h2)


def forward(packed, n_in, hid, n_out, x):
    v = unpack(packed, n_in, hid, n_out)
    o, _ = network(v, x)
    return o * v["scale"]


def loss_and_grad(packed, n_in, hid, n_out, x, t):
    """Batch loss and its gradient with respect to the trained part (W1..b3),
    flattened in packed order."""
    v = unpack(packed, n_in, hid, n_out)
    o, (xn, z1, h1, z2, h2) = network(v, x)
    diff = o - np.asarray(t, dtype=np.float64) / v["scale"]
    count = diff.size
    loss = float(np.sum(diff ** 2) / count)
    dO = 2.0 * diff / count
    gW3 = dO.T @ h2
    gb3 = dO.sum(axis=0)
    dZ2 = (dO @ v["W3"]) * silu_d(z2)
    gW2 = dZ2.T @ h1
    gb2 = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ v["W2"]) * silu_d(z1)
    gW1 = dZ1.T @ xn
    gb1 = dZ1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def train_step(packed, m, v_mom, n_in, hid, n_out, x, t, lr, step, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step; returns (packed', m', v', loss)."""
    off, _ = layout(n_in, hid, n_out)
    begin = off["W1"][0]
    loss, g = loss_and_grad(packed, n_in, hid, n_out, x, t)
    m = b1 * np.asarray(m, dtype=np.float64) + (1.0 - b1) * g
    v_mom = b2 * np.asarray(v_mom, dtype=np.float64) + (1.0 - b2) * g * g
    p = np.array(packed, dtype=np.float64)
    mhat = m / (1.0 - b1 ** step)
    vhat = v_mom / (1.0 - b2 ** step)
    p[begin:] -= lr * mhat / (np.sqrt(vhat) + eps)
    return p, m, v_mom, loss
