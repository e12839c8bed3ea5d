"""Surrogate training products on the tensor cores (pic_mlp_set_training): full-batch
gradients of every member against the FP64 reference (oracle/mlp.py) within the rounding
of BF16 operands, on a ragged batch; training that lowers the loss like the FP32 path,
reproducibly; and the width limit."""
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


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_tensor_core_gradients_match_reference(env):
    """BF16 operands carry 8 significant bits: each product's relative error is of order
    2^-9 per operand, compounded over five layers forward and back; 3% in the Frobenius
    norm of every layer's gradient bounds it with room, while a transposed operand or a
    wrong member stride gives O(1) errors."""
    pic, torch = env
    E = 3
    m = pic.pic_mlp_create(E, SIZES, 128)
    pic.pic_mlp_set_training(m, True)
    nets = members(E, SIZES, seed=21)
    pic.pic_mlp_params_set(m, np.stack([flat(W, b) for W, b in nets]))
    rng = np.random.default_rng(22)
    x = rng.uniform(-1, 1, (100, 6))
    t = rng.normal(0, 0.5, (100, 33))
    X = torch.tensor(x, dtype=torch.float32, device="cuda")
    T = torch.tensor(t, dtype=torch.float32, device="cuda")
    g, loss = pic.pic_mlp_grad(m, X, T)
    x32 = x.astype(np.float32).astype(np.float64)
    t32 = t.astype(np.float32).astype(np.float64)
    for e, (W, b) in enumerate(nets):
        W = [w.astype(np.float32).astype(np.float64) for w in W]
        b = [v.astype(np.float32).astype(np.float64) for v in b]
        y, cache = mlp.forward(W, b, x32)
        dW, db = mlp.backward(W, cache, y, t32)
        gW, gb = unflat(g[e], SIZES)
        for l in range(len(W)):
            assert _rel(gW[l], dW[l]) < 0.03, (e, l, _rel(gW[l], dW[l]))
            assert _rel(gb[l], db[l]) < 0.03, (e, l, _rel(gb[l], db[l]))
        assert abs(loss[e] / mlp.loss(y, t32) - 1.0) < 0.01


def test_tensor_core_training_lowers_the_loss_reproducibly(env):
    pic, torch = env
    rng = np.random.default_rng(13)
    x = rng.uniform(-1, 1, (512, 6))
    t = np.concatenate([np.sin(x @ rng.normal(size=(6, 32))), (x ** 2).sum(1, keepdims=True)], 1)
    X = torch.tensor(x, dtype=torch.float32, device="cuda")
    T = torch.tensor(t, dtype=torch.float32, device="cuda")
    out = {}
    for tc in (False, True, True):
        m = pic.pic_mlp_create(2, SIZES, 128)
        pic.pic_mlp_params_set(m, np.stack([flat(W, b) for W, b in members(2, SIZES, seed=14)]))
        pic.pic_mlp_set_training(m, False)
        _, loss0 = pic.pic_mlp_grad(m, X[:128], T[:128])
        pic.pic_mlp_set_training(m, tc)
        pic.pic_mlp_train(m, X, T, batch=128, steps=300, lr=1e-3, seed=5)
        pic.pic_mlp_set_training(m, False)
        _, loss1 = pic.pic_mlp_grad(m, X[:128], T[:128])
        out.setdefault(tc, []).append((pic.pic_mlp_params_get(m), loss0, loss1))
    (p32, a0, a1), = out[False]
    (p1, b0, b1), (p2, _, _) = out[True]
    assert np.all(b1 < 0.2 * b0)
    assert np.all(b1 < 1.5 * a1)                 # as good as FP32 training, near enough
    assert np.abs(p1 - p2).max() <= 1e-6 * np.abs(p1).max()


def test_tensor_core_training_needs_narrow_layers(env):
    pic, torch = env
    m = pic.pic_mlp_create(1, (6, 300, 3), 64)
    with pytest.raises(pic.PicError) as e:
        pic.pic_mlp_set_training(m, True)
    assert e.value.status == pic.PIC_ERR_ARG
