"""Surrogate host logic: the ringing-frequency estimator on synthetic power records with a
known tone, and the network targets' layout (arrival power, window ratios, frequency)
against the envelope it encodes."""
import numpy as np

from paper_1701_03784_gb300 import surrogate as S


def test_ringing_frequency_finds_the_tone_below_the_band_limit():
    """A tone on a sloping mean level, with a stronger one above the 100 GHz band limit (the
    mesh's own noise band), over 1280 samples 0.8 ps apart (1.02 ns): the estimate is
    within 0.1% of the tone, off the 1 GHz grid of the record's own spectrum."""
    dt = 8e-13
    t = np.arange(1280) * dt
    tones = np.array([4.7e9, 8.31e9, 13.7e9, 21.9e9, 47.05e9])
    rows = np.array([5.0 + 2e9 * t + np.cos(2 * np.pi * f * t + 0.3) + 3.0 * np.cos(2 * np.pi * 180e9 * t)
                     for f in tones])
    f = S.ringing_frequency(rows, dt)
    assert np.all(np.abs(f / tones - 1.0) < 1e-3), f / tones - 1.0
    # without the band limit the out-of-band tone wins; below f_min the slope's leakage
    # is not a tone
    assert np.all(S.ringing_frequency(rows, dt, f_min=0.0) > 0)
    assert np.all(np.abs(S.ringing_frequency(rows, dt, f_max=300e9) / 180e9 - 1.0) < 1e-3)


def test_targets_encode_the_envelope():
    rng = np.random.default_rng(3)
    env = rng.uniform(0.1, 2.0, (7, S.N_ENV))
    env[:, S.N_ARRIVAL:] -= 1.5           # the ringing's flux runs both ways
    freq = rng.uniform(5e9, 20e9, 7)
    current = rng.uniform(1e3, 5e3, 7)
    Y = S.targets(env, freq, current)
    assert Y.shape == (7, S.N_OUT)
    arrival = env[:, :S.N_ARRIVAL].mean(1)
    assert np.allclose(10.0 ** Y[:, 0] * (current / 1e3) ** 2, arrival, rtol=1e-12)
    assert np.allclose(S.arrival_power(Y, current), arrival, rtol=1e-12)
    # relative errors of the power the gate sees are those of the arrival power
    assert np.allclose(S.Ensemble.power(Y) / S.Ensemble.power(Y[::-1]),
                       (arrival / current ** 2) / (arrival / current ** 2)[::-1], rtol=1e-12)
    assert np.allclose(S.envelope(Y, current), env, rtol=1e-12, atol=1e-12)
    assert np.allclose(Y[:, -1], freq * 1e-9, rtol=1e-12)
    # window means of a transposed record (the port record's layout) come out column-major;
    # the targets are row-major all the same (the training copies assume it)
    YF = S.targets(np.asfortranarray(env), freq, current)
    assert YF.flags["C_CONTIGUOUS"] and np.array_equal(YF, Y)


def test_calibrated_gate_bounds_the_calibration_errors():
    spread = np.array([0.01, 0.02, 0.03, 0.04, 0.05])
    err = np.array([0.01, 0.03, 0.02, 0.045, 0.01])
    tau = S.Ensemble.calibrate(spread, err, target=0.05, margin=0.8)
    assert tau == 0.03
    assert S.Ensemble.calibrate(spread, np.full(5, 0.5)) == 0.0
