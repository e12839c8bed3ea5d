"""Surrogate mechanics on the GPU: an ensemble trained (by the library's kernels) on a
smooth function of the 6 inputs answers in-distribution queries accurately where its
members agree, and its spread grows far outside the training range, which is what sends a
query back to the simulation; and the batched-simulation outputs have the expected form."""
import numpy as np
import pytest

from workloads.bwo import EPS0, MU0, C0, QE, ME

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1701_03784_gb300 as pkg
    pkg.build()
    from paper_1701_03784_gb300 import pic, surrogate
    return pic, surrogate


def _target(x):
    """Smooth stand-in outputs: 32 log-energies and a frequency."""
    s = np.linspace(0, 1, 32)
    amp = 1.0 + 0.5 * x[:, :1] + 0.3 * x[:, 1:2] * x[:, 2:3]
    env = -3.0 + amp * s + 0.2 * np.sin(np.pi * (x[:, 3:4] + s)) + 0.1 * x[:, 4:5] * x[:, 5:6]
    freq = 10.0 + 2.0 * x[:, 5:6]
    return np.concatenate([env, freq], 1)


def test_ensemble_answers_in_range_and_flags_extrapolation(env):
    pic, S = env
    rng = np.random.default_rng(31)
    X = rng.uniform(-1, 1, (2048, 6))
    ens = S.Ensemble(5, S.SIZES, max_batch=256, seed=32)
    ens.fit(X, _target(X), steps=3000, batch=128, lr=1e-3, seed=33)
    Xin = rng.uniform(-0.9, 0.9, (256, 6))
    mean, ok, spread_in = ens.answer(Xin, tol=0.05)
    P = S.Ensemble.power(_target(Xin))
    err = np.abs(S.Ensemble.power(mean) - P) / P
    assert ok.mean() >= 0.5
    assert np.median(err[ok]) <= 0.05
    Xout = rng.uniform(2.5, 3.5, (256, 6))
    _, ok_out, spread_out = ens.answer(Xout, tol=0.05)
    assert np.median(spread_out) > 3 * np.median(spread_in)
    assert ok_out.mean() < ok.mean()


def test_batch_outputs_of_two_small_instances(env):
    pic, S = env
    from workloads.sweep import sweep_instance, WEIGHT, R0
    ins = []
    for i in (0, 1):
        x = sweep_instance(i, scale=0.002, mesh_scale=0.1)
        x["out_z"] = x["sws"][0]
        x["probe"] = (x["sws"][0] + 1.5 * x["params"]["period"], 0.7 * (R0 - x["params"]["depth"]))
        ins.append(x)
    env_, freq = S.batch_outputs(ins, 1.0e-13, 2.5, 256, 8, QE, ME, WEIGHT, EPS0, MU0, C0)
    assert env_.shape == (2, 32) and freq.shape == (2,)
    assert np.all(np.isfinite(env_)) and np.all(freq > 0)
    # the beam's field builds up from zero: energy grows over the run
    assert np.all(env_[:, -1] > env_[:, 0])
