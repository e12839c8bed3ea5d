"""FP64 reference of the surrogate network (test infrastructure: imported by tests/ only).

A multilayer perceptron maps the 6 normalised sweep parameters (ripple depth, period,
number of periods, beam voltage, beam current, guide field) through 4 hidden layers of
256 units with GELU (tanh form) to 33 outputs (32 samples of the output envelope and the
dominant frequency), trained on mean-squared error.  Written out plainly: every layer is
z = x W^T + b, a = gelu(z); the backward pass applies the chain rule layer by layer.  It is
pinned by finite differences and by closed forms in tests/test_oracle_mlp.py.
"""
import numpy as np

SIZES = (6, 256, 256, 256, 256, 33)
C_GELU = np.sqrt(2.0 / np.pi)


def gelu(z):
    """0.5 z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3)))"""
    return 0.5 * z * (1.0 + np.tanh(C_GELU * (z + 0.044715 * z ** 3)))


def gelu_grad(z):
    t = np.tanh(C_GELU * (z + 0.044715 * z ** 3))
    dt = (1.0 - t * t) * C_GELU * (1.0 + 3 * 0.044715 * z * z)
    return 0.5 * (1.0 + t) + 0.5 * z * dt


def init(seed, sizes=SIZES):
    """Weights W_l (n_out x n_in) ~ U(-1/sqrt(n_in), 1/sqrt(n_in)), biases zero."""
    rng = np.random.default_rng(seed)
    Ws, bs = [], []
    for k, n in zip(sizes[:-1], sizes[1:]):
        lim = 1.0 / np.sqrt(k)
        Ws.append(rng.uniform(-lim, lim, (n, k)))
        bs.append(np.zeros(n))
    return Ws, bs


def forward(Ws, bs, x):
    """Returns the output and the per-layer (input, pre-activation) pairs."""
    cache = []
    a = x
    L = len(Ws)
    for l in range(L):
        z = a @ Ws[l].T + bs[l]
        cache.append((a, z))
        a = gelu(z) if l < L - 1 else z
    return a, cache


def loss(y, t):
    """Mean over samples and outputs of the squared error."""
    return np.mean((y - t) ** 2)


def backward(Ws, cache, y, t):
    """Gradients (dW_l, db_l) of loss(y, t) with respect to every layer's parameters."""
    L = len(Ws)
    g = 2.0 * (y - t) / y.size          # d loss / d y
    dWs, dbs = [None] * L, [None] * L
    for l in range(L - 1, -1, -1):
        a, z = cache[l]
        if l < L - 1:
            g = g * gelu_grad(z)        # through the activation of layer l
        dWs[l] = g.T @ a
        dbs[l] = g.sum(0)
        g = g @ Ws[l]                   # to the layer's input
    return dWs, dbs


def adam(params, grads, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update in place (bias-corrected moments)."""
    for p, g, mm, vv in zip(params, grads, m, v):
        mm *= b1
        mm += (1 - b1) * g
        vv *= b2
        vv += (1 - b2) * g * g
        mh = mm / (1 - b1 ** step)
        vh = vv / (1 - b2 ** step)
        p -= lr * mh / (np.sqrt(vh) + eps)
