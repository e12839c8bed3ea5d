"""Host-side helpers of the package: the graded absorbing-layer profile (ports.py) and the
cold test's frequency fit (coldtest.py).  CPU only."""
import math

import numpy as np
import pytest

import workloads as W


def test_graded_layer_profile():
    from paper_1701_03784_gb300 import ports
    nodes, tris, be, bt = W.meshes.rect_mesh(10.0, 1.0, 800, 3)
    en = np.array(sorted({tuple(sorted((int(t[i]), int(t[(i + 1) % 3])))) for t in tris
                          for i in range(3)}))
    smax = ports.sigma_max_for(1e-4, 2.0, 3, eps0=2.0, c=3.0)
    assert smax == pytest.approx(4 * math.log(1e4) * 2.0 * 3.0 / 4.0)
    se, sm = ports.graded_layer(nodes, en, tris, 8.0, 10.0, smax, 3, eps0=2.0, mu0=5.0)
    ze = 0.5 * (nodes[en[:, 0], 0] + nodes[en[:, 1], 0])
    assert np.all(se[ze <= 8.0] == 0.0) and np.all(se[ze > 8.0] > 0.0)
    assert np.allclose(se[ze > 8.0], smax * ((ze[ze > 8.0] - 8.0) / 2.0) ** 3)
    zf = nodes[tris][:, :, 0].mean(1)
    # matched: sigma_m / sigma_e = mu0 / eps0 at the same z
    assert np.allclose(sm, smax * np.clip((zf - 8.0) / 2.0, 0, 1) ** 3 * 5.0 / 2.0)
    # a layer on the left grades the other way
    se2, _ = ports.graded_layer(nodes, en, tris, 2.0, 0.0, smax, 3)
    assert np.all(se2[ze >= 2.0] == 0.0) and se2[np.argmin(ze)] > 0.0


def test_cold_test_frequency_fit():
    pytest.importorskip("scipy")
    from paper_1701_03784_gb300 import coldtest
    t = np.arange(4000) * 2.5e-13
    f1, f2 = 7.3e9, 24.1e9
    a = 3.0 * np.cos(2 * np.pi * f1 * t + 0.4) + 0.5 * np.sin(2 * np.pi * f2 * t) + 0.1
    assert coldtest._frequency(t, a) == pytest.approx(f1, rel=1e-7)
