"""Shared helpers of the surrogate-network tests: the reference network's parameters in
the library's layout (per member, W_l row-major then b_l)."""
import numpy as np

from oracle import mlp


def flat(Ws, bs):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in zip(Ws, bs)])


def unflat(p, sizes):
    Ws, bs, o = [], [], 0
    for k, n in zip(sizes[:-1], sizes[1:]):
        Ws.append(p[o:o + n * k].reshape(n, k))
        o += n * k
        bs.append(p[o:o + n])
        o += n
    return Ws, bs


def members(n_members, sizes, seed=0, bias_scale=0.1):
    """Reference parameters of n_members networks (small random biases)."""
    rng = np.random.default_rng(seed + 1000)
    out = []
    for e in range(n_members):
        Ws, bs = mlp.init(seed + e, sizes)
        bs = [rng.normal(0, bias_scale, b.shape) for b in bs]
        out.append((Ws, bs))
    return out
