"""Pins of the FP64 surrogate-network reference: GELU against its closed form and limits,
the backward pass against central finite differences of the loss, a network without
hidden nonlinearity against the plain matrix product, and Adam's first step against its
closed form (a step of -lr sign(g))."""
import math

import numpy as np

from oracle import mlp


def test_gelu_closed_form_and_limits():
    z = np.array([-3.0, -1.0, 0.0, 0.5, 2.0])
    ref = [0.5 * x * (1 + math.tanh(math.sqrt(2 / math.pi) * (x + 0.044715 * x ** 3)))
           for x in z]
    assert np.allclose(mlp.gelu(z), ref, rtol=0, atol=1e-15)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    big = np.array([30.0, -30.0])
    assert np.allclose(mlp.gelu(big), [30.0, 0.0], atol=1e-12)
    # derivative against central differences
    h = 1e-6
    zz = np.linspace(-4, 4, 41)
    fd = (mlp.gelu(zz + h) - mlp.gelu(zz - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(zz), fd, rtol=0, atol=1e-8)


def test_backward_matches_finite_differences():
    sizes = (6, 7, 5, 4)
    Ws, bs = mlp.init(3, sizes)
    rng = np.random.default_rng(4)
    for b in bs:
        b += rng.normal(0, 0.1, b.shape)
    x = rng.normal(size=(9, 6))
    t = rng.normal(size=(9, 4))
    y, cache = mlp.forward(Ws, bs, x)
    dWs, dbs = mlp.backward(Ws, cache, y, t)
    h = 1e-6
    for l in range(len(Ws)):
        for (i, j) in [(0, 0), (1, 2), (len(Ws[l]) - 1, Ws[l].shape[1] - 1)]:
            Wp = [w.copy() for w in Ws]
            Wm = [w.copy() for w in Ws]
            Wp[l][i, j] += h
            Wm[l][i, j] -= h
            fd = (mlp.loss(mlp.forward(Wp, bs, x)[0], t) -
                  mlp.loss(mlp.forward(Wm, bs, x)[0], t)) / (2 * h)
            assert abs(dWs[l][i, j] - fd) < 1e-8 * max(1.0, abs(fd)), (l, i, j)
        for i in (0, len(bs[l]) - 1):
            bp = [b.copy() for b in bs]
            bm = [b.copy() for b in bs]
            bp[l][i] += h
            bm[l][i] -= h
            fd = (mlp.loss(mlp.forward(Ws, bp, x)[0], t) -
                  mlp.loss(mlp.forward(Ws, bm, x)[0], t)) / (2 * h)
            assert abs(dbs[l][i] - fd) < 1e-8 * max(1.0, abs(fd)), (l, i)


def test_single_layer_is_the_affine_map():
    Ws, bs = mlp.init(5, (6, 3))
    bs[0][:] = [0.5, -1.0, 2.0]
    x = np.arange(12.0).reshape(2, 6)
    y, _ = mlp.forward(Ws, bs, x)
    assert np.allclose(y, x @ Ws[0].T + bs[0], atol=1e-14)


def test_adam_first_step_is_signed_learning_rate():
    p = [np.array([1.0, 2.0, 3.0])]
    g = [np.array([0.3, -2.0, 1e-3])]
    m = [np.zeros(3)]
    v = [np.zeros(3)]
    mlp.adam(p, g, m, v, 1, lr=0.01, eps=0.0)
    assert np.allclose(p[0], [0.99, 2.01, 2.99], atol=1e-15)
