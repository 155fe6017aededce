"""Plain FP64 NumPy MLP of the learned surrogate (test infrastructure).

Network 24 -> 64 -> 64 -> 6 with tanh hidden activations and a linear output,
mean-squared-error loss over the 6 outputs, Adam (Kingma & Ba) with the
bias-corrected moments.  The paper has no learned part; this is the reading
of the surrogate network (activation and optimizer are not given anywhere).
Parameters are kept in one flat vector in the order W1 [64,24], b1 [64],
W2 [64,64], b2 [64], W3 [6,64], b3 [6] (row-major), the layout the CUDA
kernels use.

Pins (tests/test_oracle_mlp.py): gradients equal central finite differences;
one Adam step equals the textbook update written out elementwise.
"""
import numpy as np

SIZES = (24, 64, 64, 6)


def n_params(sizes=SIZES):
    return sum(sizes[i + 1] * sizes[i] + sizes[i + 1] for i in range(len(sizes) - 1))


def unpack(theta, sizes=SIZES):
    out, o = [], 0
    for i in range(len(sizes) - 1):
        r, c = sizes[i + 1], sizes[i]
        W = theta[o:o + r * c].reshape(r, c)
        o += r * c
        b = theta[o:o + r]
        o += r
        out.append((W, b))
    return out


def init(rng, sizes=SIZES):
    """Glorot-uniform weights, zero biases."""
    parts = []
    for i in range(len(sizes) - 1):
        r, c = sizes[i + 1], sizes[i]
        lim = np.sqrt(6.0 / (r + c))
        parts += [rng.uniform(-lim, lim, r * c), np.zeros(r)]
    return np.concatenate(parts)


def forward(theta, X):
    """Outputs [n, 6] and the hidden activations."""
    layers = unpack(theta)
    acts = [X]
    h = X
    for li, (W, b) in enumerate(layers):
        z = h @ W.T + b
        h = np.tanh(z) if li < len(layers) - 1 else z
        acts.append(h)
    return h, acts


def loss(theta, X, Y):
    out, _ = forward(theta, X)
    return np.mean((out - Y) ** 2)


def grad(theta, X, Y):
    """d loss / d theta by backpropagation."""
    layers = unpack(theta)
    out, acts = forward(theta, X)
    n = X.shape[0]
    delta = 2.0 * (out - Y) / (n * Y.shape[1])
    grads = []
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        a_in = acts[li]
        gW = delta.T @ a_in
        gb = delta.sum(axis=0)
        grads.append((gW, gb))
        if li > 0:
            delta = (delta @ W) * (1.0 - acts[li] ** 2)
    grads = grads[::-1]
    return np.concatenate([np.concatenate([gW.reshape(-1), gb]) for gW, gb in grads])


def adam_step(theta, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t counts from 1)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
