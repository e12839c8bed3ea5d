"""SPAI pattern / drop-tolerance sweep (Sec. 3.1 leaves both open): the library's M, stable
step and residual ||star_eps_ff M - I|| against the oracle across the sweep, and the
oracle's residual falling as the pattern grows.  Host-only (CPU)."""
import numpy as np
import pytest

import workloads as W
from oracle.operators import Mesh, hodge_eps, hodge_mu_inv, spai, dt_stable

SWEEP = [(1, 0.0), (1, 1e-2), (2, 1e-3), (3, 1e-4)]


@pytest.fixture(scope="module")
def pic():
    import paper_1701_03784_gb300 as pkg
    pkg.build()
    from paper_1701_03784_gb300 import pic as p
    return p


@pytest.fixture(scope="module")
def cavity():
    nodes, tris, be, bt = W.cavity_mesh(n_tri=600, seed=3)
    om = Mesh(nodes, tris, be, bt)
    return (nodes, tris, be, bt), om, hodge_eps(om, 1.0)


def _residual(om, A, M):
    Aff = A[om.free][:, om.free]
    R = (Aff @ M).toarray() - np.eye(len(om.free))
    return np.linalg.norm(R) / np.sqrt(len(om.free)), np.abs(R).max()


@pytest.mark.parametrize("level,tau", SWEEP)
def test_library_spai_matches_oracle_across_the_sweep(pic, cavity, level, tau):
    arrays, om, A = cavity
    m = pic.pic_mesh_create(*arrays)
    dt = pic.pic_spai_build(m, level, tau)
    fe, ip, ix, vv = pic.pic_spai_get(m)
    M = spai(om, A, level, tau).tocsr()
    M.sort_indices()
    assert np.array_equal(ip, M.indptr) and np.array_equal(ix, M.indices)
    assert np.allclose(vv, M.data, rtol=1e-9, atol=1e-12 * np.abs(M.data).max())
    dt_o, _ = dt_stable(om, M, hodge_mu_inv(om, 1.0))
    assert abs(dt - dt_o) <= 1e-9 * dt_o
    info = pic.pic_spai_info(m)
    rms, mx = _residual(om, A, M)
    assert info["nnz"] == M.nnz
    assert info["residual_rms"] == pytest.approx(rms, rel=1e-8)
    assert info["residual_max"] == pytest.approx(mx, rel=1e-8)
    pic.pic_mesh_destroy(m)


def test_oracle_spai_residual_falls_as_the_pattern_grows(cavity):
    """Nested patterns: each level's least-squares columns can only fit better; with no
    dropping the residual falls by more than half per level on this mesh.  (The full
    pattern giving the inverse is pinned on a small mesh in test_oracle_operators.py.)"""
    arrays, om, A = cavity
    res, nnz = [], []
    for level in (1, 2, 3):
        M = spai(om, A, level, 0.0).tocsr()
        res.append(_residual(om, A, M)[0])
        nnz.append(M.nnz)
    assert res[1] < 0.5 * res[0] and res[2] < 0.5 * res[1]
    assert nnz[0] < nnz[1] < nnz[2]


def test_spai_info_needs_a_built_spai(pic, cavity):
    arrays, _, _ = cavity
    m = pic.pic_mesh_create(*arrays)
    with pytest.raises(pic.PicError) as e:
        pic.pic_spai_info(m)
    assert e.value.status == pic.PIC_ERR_STATE
    pic.pic_mesh_destroy(m)
