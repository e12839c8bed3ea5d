"""Surrogate network inference on the tensor cores (tcgen05, BF16 operands, FP32
accumulation in TMEM) against the FP64 reference and the FP32 path, for every member, a
ragged last tile and a chunk of many tiles."""
import numpy as np
import pytest

from oracle import mlp
from tests.mlp_util import flat, members

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


@pytest.mark.parametrize("n", [1, 200, 4100])
def test_tensor_core_forward_matches_reference(env, n):
    pic, torch = env
    E = 5
    m = pic.pic_mlp_create(E, SIZES, 256)
    nets = members(E, SIZES, seed=21)
    pic.pic_mlp_params_set(m, np.stack([flat(W, b) for W, b in nets]))
    x = np.random.default_rng(22 + n).uniform(-1, 1, (n, 6))
    X = torch.tensor(x, dtype=torch.float32, device="cuda")
    Yt = pic.pic_mlp_forward(m, X, tensor_cores=True).cpu().numpy()
    Yf = pic.pic_mlp_forward(m, X, tensor_cores=False).cpu().numpy()
    for e, (W, b) in enumerate(nets):
        y, _ = mlp.forward(W, b, x)
        scale = np.abs(y).max()
        # BF16 operands (8 significant bits) over 5 layers, FP32 accumulation
        assert np.abs(Yt[e] - y).max() <= 3e-2 * scale, e
        assert np.abs(Yf[e] - y).max() <= 1e-5 * scale, e
        assert np.sqrt(np.mean((Yt[e] - y) ** 2)) <= 1e-2 * np.sqrt(np.mean(y ** 2)), e


@pytest.mark.parametrize("sizes", [(6, 96, 48, 200, 33), (3, 16, 5)])
def test_tensor_core_forward_uneven_widths(env, sizes):
    """Widths that are not multiples of the 64-row weight slices: a layer's last slice
    has 32, 16 or 48 rows (padded widths 96, 48, 208), and a one-hidden-layer network."""
    pic, torch = env
    E, n = 3, 700
    m = pic.pic_mlp_create(E, sizes, 256)
    nets = members(E, sizes, seed=31)
    pic.pic_mlp_params_set(m, np.stack([flat(W, b) for W, b in nets]))
    x = np.random.default_rng(32).uniform(-1, 1, (n, sizes[0]))
    X = torch.tensor(x, dtype=torch.float32, device="cuda")
    Yt = pic.pic_mlp_forward(m, X, tensor_cores=True).cpu().numpy()
    for e, (W, b) in enumerate(nets):
        y, _ = mlp.forward(W, b, x)
        scale = np.abs(y).max()
        assert np.abs(Yt[e] - y).max() <= 3e-2 * scale, e
        assert np.sqrt(np.mean((Yt[e] - y) ** 2)) <= 1e-2 * np.sqrt(np.mean(y ** 2)), e
