"""Pins of the oracle's mesh operators against facts fixed by the paper and by mathematics,
not by the oracle itself.  CPU only."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle.operators import (Mesh, hodge_eps, hodge_mu_inv, local_hodge_eps, spai,
                              dt_stable, curl_curl)
from oracle.particles import barycentric


def _meshes():
    return [W.two_triangle_mesh(), W.four_triangle_mesh(), W.cavity_mesh(n_tri=300, seed=5),
            W.bwo_small_mesh(n_tri=3000, seed=9)]


def _grad_by_solve(p):
    """grad(lambda) of one triangle from the 3x3 system [1; x; y] lambda = [1; x; y]
    (independent of the oracle's closed form)."""
    A = np.array([[1.0, 1.0, 1.0], p[:, 0], p[:, 1]])
    inv = np.linalg.inv(A)
    return inv[:, 1:]                                        # rows k: (dl_k/dz, dl_k/drho)


def _duffy_rule(n):
    """Quadrature on the reference triangle (0,0),(1,0),(0,1) from an n x n Gauss
    product rule on the square through the collapsed (Duffy) map; exact for degree
    2n-2 polynomials."""
    x, w = np.polynomial.legendre.leggauss(n)
    x = 0.5 * (x + 1)
    w = 0.5 * w
    pts, wts = [], []
    for xi, wi in zip(x, w):
        for eta, we in zip(x, w):
            pts.append((xi, (1 - xi) * eta))
            wts.append(wi * we * (1 - xi))
    return np.array(pts), np.array(wts)


@pytest.mark.parametrize("mi", range(4))
def test_incidence_identities(mi):
    """D_div D_curl^T = 0 (Sec. 3.5.2); Euler's formula; each interior edge bounds two
    faces with opposite orientation (App. D)."""
    m = Mesh(*_meshes()[mi])
    Z = (m.Ddiv @ m.Dcurl.T).tocoo()
    assert np.all(Z.data == 0)
    assert m.N0 - m.N1 + m.N2 == 1
    s = np.asarray(m.Dcurl.sum(0)).ravel()
    interior = m.edge_tag == 0
    assert np.all(s[interior] == 0)
    assert np.all(np.abs(s[~interior]) == 1)
    assert np.all(np.abs(m.Dcurl.data) == 1) and np.all(np.abs(m.Ddiv.data) == 1)


@pytest.mark.parametrize("mi", range(4))
def test_gradients_and_area(mi):
    m = Mesh(*_meshes()[mi])
    for t in range(0, m.N2, max(1, m.N2 // 50)):
        p = m.nodes[m.tris[t]]
        assert np.allclose(m.grad[t], _grad_by_solve(p), rtol=1e-12, atol=1e-12 / m.area[t])
        a2 = (p[1, 0] - p[0, 0]) * (p[2, 1] - p[0, 1]) - (p[2, 0] - p[0, 0]) * (p[1, 1] - p[0, 1])
        assert a2 > 0 and abs(0.5 * a2 - m.area[t]) <= 1e-14 * m.area[t]


def test_whitney_pairing():
    """<sigma_i, w_j> = delta_ij (App. A): the line integral of W1_j along edge i,
    oriented low -> high node index, is 1 for i = j and 0 otherwise."""
    m = Mesh(*W.cavity_mesh(n_tri=200, seed=3))
    x, w = np.polynomial.legendre.leggauss(4)
    x, w = 0.5 * (x + 1), 0.5 * w
    for t in range(0, m.N2, 7):
        G = _grad_by_solve(m.nodes[m.tris[t]])
        for ki in range(3):
            a_i, b_i = m.edge_tail_head(t, ki)
            pa, pb = m.nodes[m.tris[t, a_i]], m.nodes[m.tris[t, b_i]]
            for kj in range(3):
                a, b = m.edge_tail_head(t, kj)
                val = 0.0
                for xq, wq in zip(x, w):
                    q = pa + xq * (pb - pa)
                    lam = barycentric(m, np.array([t]), np.array([q[0]]), np.array([q[1]]))[0]
                    Wv = lam[a] * G[b] - lam[b] * G[a]
                    val += wq * Wv @ (pb - pa)
                assert abs(val - (1.0 if ki == kj else 0.0)) < 1e-12


@pytest.mark.parametrize("mi", range(4))
def test_hodge_eps_by_quadrature(mi):
    """[star_eps]_ij = eps0 int rho W_i . W_j dz drho (App. B, defining integral), by a
    Duffy-Gauss rule with gradients from a linear solve."""
    m = Mesh(*_meshes()[mi])
    eps0 = 2.5
    T = local_hodge_eps(m, eps0)
    qp, qw = _duffy_rule(4)
    for t in range(0, m.N2, max(1, m.N2 // 40)):
        p = m.nodes[m.tris[t]]
        G = _grad_by_solve(p)
        J = np.array([p[1] - p[0], p[2] - p[0]]).T
        det = abs(np.linalg.det(J))
        ref = np.zeros((3, 3))
        for (s, r), wq in zip(qp, qw):
            lam = np.array([1 - s - r, s, r])
            rho = lam @ p[:, 1]
            Wk = []
            for k in range(3):
                a, b = m.edge_tail_head(t, k)
                Wk.append(lam[a] * G[b] - lam[b] * G[a])
            for i in range(3):
                for j in range(3):
                    ref[i, j] += wq * det * eps0 * rho * Wk[i] @ Wk[j]
        assert np.allclose(T[t], ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())


def test_hodge_eps_constant_rho_textbook():
    """With rho constant the edge-element mass matrix of a right isosceles triangle with
    legs h is known in closed form; shift the triangle far from the axis so that rho is
    nearly constant and compare the rho-weighted matrix divided by rho."""
    h = 1.0
    R0 = 1e9
    nodes = np.array([[0.0, R0], [h, R0], [0.0, R0 + h]])
    tris = np.array([[0, 1, 2]])
    bedges = np.array([[0, 1], [1, 2], [0, 2]])
    m = Mesh(nodes, tris, bedges, np.array([1, 1, 1]))
    T = local_hodge_eps(m, 1.0)[0] / R0
    # edges: k=0 (1->2, hypotenuse), k=1 (0->2), k=2 (0->1).  With lambda_1 = x,
    # lambda_2 = y, lambda_0 = 1 - x - y (h = 1): W_0 = (-y, x), W_1 = (y, 1 - x),
    # W_2 = (1 - y, x); the monomial integrals int x^2 = 1/12, int xy = 1/24,
    # int x = 1/6, int 1 = 1/2 give:
    ref = np.array([[1 / 6, 0.0, 0.0], [0.0, 1 / 3, 1 / 6], [0.0, 1 / 6, 1 / 3]])
    assert np.allclose(T, ref, atol=1e-7)


@pytest.mark.parametrize("mi", range(4))
def test_hodge_mu_by_quadrature(mi):
    """[star_mu^-1]_ff = (1/mu0) int rho (W2)^2 with W2 = 1/A (App. B)."""
    m = Mesh(*_meshes()[mi])
    mu0 = 0.7
    d = hodge_mu_inv(m, mu0)
    qp, qw = _duffy_rule(3)
    for t in range(0, m.N2, max(1, m.N2 // 40)):
        p = m.nodes[m.tris[t]]
        det = 2 * m.area[t]
        ref = sum(wq * det * ((1 - s - r) * p[0, 1] + s * p[1, 1] + r * p[2, 1])
                  for (s, r), wq in zip(qp, qw)) / (mu0 * m.area[t] ** 2)
        assert abs(d[t] - ref) <= 1e-13 * ref


def test_hodge_spd():
    m = Mesh(*W.cavity_mesh(n_tri=400, seed=4))
    A = hodge_eps(m).toarray()
    assert np.allclose(A, A.T, rtol=0, atol=1e-15 * np.abs(A).max())
    f = m.free
    assert np.linalg.eigvalsh(A[np.ix_(f, f)]).min() > 0
    # five nonzeros per row for interior edges (App. B)
    nnz = np.diff(hodge_eps(m).indptr)
    assert np.all(nnz[m.edge_tag == 0] == 5)


def test_spai_level0_closed_form():
    """A one-entry pattern gives the least-squares scalar m_j = A_jj / ||A_:j||^2."""
    m = Mesh(*W.cavity_mesh(n_tri=200, seed=8))
    A = hodge_eps(m)
    M = spai(m, A, level=0, drop_tol=0.0).toarray()
    Af = A[m.free][:, m.free].toarray()
    ref = np.diag(Af) / np.sum(Af * Af, 0)
    assert np.allclose(np.diag(M), ref, rtol=1e-12)
    assert np.count_nonzero(M - np.diag(np.diag(M))) == 0


def test_spai_full_pattern_is_inverse():
    """When the pattern covers every edge the least-squares problem is square: M = A^-1."""
    m = Mesh(*W.four_triangle_mesh())
    A = hodge_eps(m)
    M = spai(m, A, level=6, drop_tol=0.0).toarray()
    Af = A[m.free][:, m.free].toarray()
    assert np.allclose(M, np.linalg.inv(Af), rtol=1e-10, atol=1e-12 * np.abs(M).max())


def test_spai_quality_and_symmetry():
    m = Mesh(*W.cavity_mesh(n_tri=600, seed=2))
    A = hodge_eps(m)
    M = spai(m, A, level=2, drop_tol=1e-4)
    assert abs(M - M.T).max() == 0
    Af = A[m.free][:, m.free]
    err = sp.linalg.norm(Af @ M - sp.identity(len(m.free))) / math.sqrt(len(m.free))
    assert err < 0.05


def test_dt_stable_matches_eigensolver():
    """Power-iteration lambda_max(M K) against a dense eigensolver."""
    m = Mesh(*W.cavity_mesh(n_tri=300, seed=6))
    A = hodge_eps(m)
    M = spai(m, A)
    mu = hodge_mu_inv(m)
    dt, lam = dt_stable(m, M, mu, iters=3000)
    ev = np.linalg.eigvals((M @ curl_curl(m, mu)).toarray())
    assert abs(ev.imag).max() < 1e-6 * abs(ev.real).max()
    assert abs(lam - ev.real.max()) / ev.real.max() < 1e-3
    assert abs(dt - 2 / math.sqrt(ev.real.max())) / dt < 1e-3


def test_table1_closed_form():
    """The TM_0np closed form used for the cavity check reproduces the analytic
    frequencies printed in Table 1 (Sec. 4.1) within 0.3% (three printed digits; the
    paper does not state the value of c it used, and one row, (0,2,2), sits 0.15% off)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_tm0np.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 17
    for r in rows:
        n, p, fa = int(r[4]), int(r[5]), float(r[6])
        f = W.tm0np_omega(0.5, 1.0, n, p, c=299792458.0) / (2 * math.pi) / 1e9
        assert abs(f - fa) <= 3e-3 * fa, r   # printed to three digits
