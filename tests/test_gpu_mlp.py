"""Surrogate network on the GPU, FP32 path: forward outputs and full-batch gradients of
every ensemble member against the FP64 reference (oracle/mlp.py) at the same parameters,
and training that lowers the loss, reproducibly."""
import numpy as np
import pytest

from oracle import mlp
from tests.mlp_util import flat, unflat, members

pytestmark = pytest.mark.gpu
SIZES = (6, 256, 256, 256, 256, 33)


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1701_03784_gb300 as pkg
    pkg.build()
    from paper_1701_03784_gb300 import pic
    return pic, torch


def test_forward_and_gradients_match_reference(env):
    pic, torch = env
    E = 3
    m = pic.pic_mlp_create(E, SIZES, 128)
    nets = members(E, SIZES, seed=11)
    pic.pic_mlp_params_set(m, np.stack([flat(W, b) for W, b in nets]))
    rng = np.random.default_rng(12)
    x = rng.uniform(-1, 1, (100, 6))
    t = rng.normal(0, 0.5, (100, 33))
    X = torch.tensor(x, dtype=torch.float32, device="cuda")
    T = torch.tensor(t, dtype=torch.float32, device="cuda")
    Y = pic.pic_mlp_forward(m, X).cpu().numpy()
    g, loss = pic.pic_mlp_grad(m, X, T)
    x32 = x.astype(np.float32).astype(np.float64)
    t32 = t.astype(np.float32).astype(np.float64)
    for e, (W, b) in enumerate(nets):
        W = [w.astype(np.float32).astype(np.float64) for w in W]
        b = [v.astype(np.float32).astype(np.float64) for v in b]
        y, cache = mlp.forward(W, b, x32)
        assert np.abs(Y[e] - y).max() <= 1e-5 * np.abs(y).max(), e
        dW, db = mlp.backward(W, cache, y, t32)
        gW, gb = unflat(g[e], SIZES)
        for l in range(len(W)):
            assert np.abs(gW[l] - dW[l]).max() <= 1e-4 * np.abs(dW[l]).max(), (e, l)
            assert np.abs(gb[l] - db[l]).max() <= 1e-4 * np.abs(db[l]).max(), (e, l)
        assert abs(loss[e] - mlp.loss(y, t32)) <= 1e-5 * mlp.loss(y, t32)


def test_training_lowers_the_loss_reproducibly(env):
    pic, torch = env
    rng = np.random.default_rng(13)
    x = rng.uniform(-1, 1, (512, 6))
    # a smooth target of the inputs
    t = np.concatenate([np.sin(x @ rng.normal(size=(6, 32))), (x ** 2).sum(1, keepdims=True)], 1)
    X = torch.tensor(x, dtype=torch.float32, device="cuda")
    T = torch.tensor(t, dtype=torch.float32, device="cuda")
    runs = []
    for _ in range(2):
        m = pic.pic_mlp_create(2, SIZES, 64)
        pic.pic_mlp_params_set(m, np.stack([flat(W, b) for W, b in members(2, SIZES, seed=14)]))
        _, loss0 = pic.pic_mlp_grad(m, X[:64], T[:64])
        pic.pic_mlp_train(m, X, T, batch=64, steps=300, lr=1e-3, seed=5)
        _, loss1 = pic.pic_mlp_grad(m, X[:64], T[:64])
        runs.append((pic.pic_mlp_params_get(m), loss0, loss1))
    (p1, a0, a1), (p2, b0, b1) = runs
    assert np.all(a1 < 0.2 * a0)
    # same seed, same draws: the same parameters up to the order of float atomics in the
    # loss (the updates themselves have no atomics)
    assert np.abs(p1 - p2).max() <= 1e-6 * np.abs(p1).max()
