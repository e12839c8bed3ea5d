"""Mesh operators of the mixed E-B FETD scheme, FP64 numpy/scipy.  Test infrastructure.

Coordinates: the meridian plane with x = z, y = rho.  Then dz^drho = dx^dy and the
out-of-plane unit vector x-hat cross y-hat is +phi-hat, so a counter-clockwise
traversal in (z, rho) is the positive orientation of a face (Sec. 2.1: B = B_phi dz^drho).
"""
import math

import numpy as np
import scipy.sparse as sp

BC_INTERIOR, BC_PEC, BC_AXIS, BC_ABSORB = 0, 1, 2, 3


class Mesh:
    """Triangle mesh of the meridian plane with its incidence structure.

    * triangles are re-oriented counter-clockwise (swap of local nodes 1 and 2);
    * edges are node pairs (lo, hi), oriented from the lower to the higher node index
      (App. D), numbered in lexicographic order of (lo, hi);
    * local edge k of a triangle joins local nodes (k+1)%3 and (k+2)%3 (it is opposite
      local node k); ``nbr[t,k]`` is the triangle across it or -1;
    * ``dcurl_sign[t,k]`` = +1 when the edge orientation agrees with the
      counter-clockwise boundary of the triangle, else -1 (rows of D_curl, Sec. 3.1).
    """

    def __init__(self, nodes, tris, bedges, btags):
        self.nodes = np.asarray(nodes, np.float64)
        tris = np.array(tris, np.int64)
        p = self.nodes[tris]
        s2 = ((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1])
              - (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1]))
        if np.any(s2 == 0.0):
            raise ValueError("degenerate triangle")
        neg = s2 < 0
        tris[neg] = tris[neg][:, [0, 2, 1]]
        self.tris = tris
        N0, N2 = len(self.nodes), len(tris)
        self.N0, self.N2 = N0, N2

        # local edge k joins local nodes (k+1)%3 -> (k+2)%3 along the ccw boundary
        i1 = tris[:, [1, 2, 0]]
        i2 = tris[:, [2, 0, 1]]
        lo = np.minimum(i1, i2)
        hi = np.maximum(i1, i2)
        key = (lo * N0 + hi).ravel()
        ukey, inv = np.unique(key, return_inverse=True)
        self.edge_nodes = np.stack([ukey // N0, ukey % N0], 1)
        self.N1 = len(ukey)
        self.tri_edges = inv.reshape(N2, 3)
        self.dcurl_sign = np.where(i1 < i2, 1, -1).astype(np.int64)

        # triangles on each edge -> neighbours
        et = -np.ones((self.N1, 2), np.int64)
        el = -np.ones((self.N1, 2), np.int64)
        cnt = np.zeros(self.N1, np.int64)
        for t in range(N2):
            for k in range(3):
                e = self.tri_edges[t, k]
                if cnt[e] >= 2:
                    raise ValueError("edge shared by more than two triangles")
                et[e, cnt[e]] = t
                el[e, cnt[e]] = k
                cnt[e] += 1
        self.edge_tris = et
        self.nbr = -np.ones((N2, 3), np.int64)
        both = cnt == 2
        self.nbr[et[both, 0], el[both, 0]] = et[both, 1]
        self.nbr[et[both, 1], el[both, 1]] = et[both, 0]

        # boundary tags: every edge with one triangle must be listed in bedges
        self.edge_tag = np.zeros(self.N1, np.int64)
        bedges = np.asarray(bedges, np.int64)
        bkey = np.minimum(bedges[:, 0], bedges[:, 1]) * N0 + np.maximum(bedges[:, 0], bedges[:, 1])
        pos = np.searchsorted(ukey, bkey)
        if np.any(pos >= self.N1) or np.any(ukey[np.minimum(pos, self.N1 - 1)] != bkey):
            raise ValueError("boundary edge not in mesh")
        if np.any(cnt[pos] != 1):
            raise ValueError("listed boundary edge is interior")
        self.edge_tag[pos] = np.asarray(btags, np.int64)
        if np.any(self.edge_tag[cnt == 1] == 0):
            raise ValueError("mesh boundary edge without a tag")
        self.tri_btag = self.edge_tag[self.tri_edges]

        # geometry: area and grad(lambda_k) = (y_{k+1} - y_{k+2}, x_{k+2} - x_{k+1}) / (2A)
        p = self.nodes[tris]
        self.area = 0.5 * np.abs(s2)
        x, y = p[:, :, 0], p[:, :, 1]
        g = np.zeros((N2, 3, 2))
        for k in range(3):
            a, b = (k + 1) % 3, (k + 2) % 3
            g[:, k, 0] = (y[:, a] - y[:, b]) / (2 * self.area)
            g[:, k, 1] = (x[:, b] - x[:, a]) / (2 * self.area)
        self.grad = g

        # incidence matrices (Sec. 3.1 / App. D); D_div: +1 at an edge's tail (lower
        # node index), -1 at its head, so D_div J is the net current leaving a node.
        rows = np.repeat(np.arange(N2), 3)
        self.Dcurl = sp.csr_matrix((self.dcurl_sign.ravel().astype(float),
                                    (rows, self.tri_edges.ravel())), shape=(N2, self.N1))
        en = self.edge_nodes
        self.Ddiv = sp.csr_matrix(
            (np.concatenate([np.ones(self.N1), -np.ones(self.N1)]),
             (np.concatenate([en[:, 0], en[:, 1]]), np.concatenate([np.arange(self.N1)] * 2))),
            shape=(N0, self.N1))

        self.free = np.flatnonzero(self.edge_tag != BC_PEC)      # E degrees of freedom
        pec_nodes = np.unique(self.edge_nodes[self.edge_tag == BC_PEC].ravel())
        self.node_on_pec = np.zeros(N0, bool)
        self.node_on_pec[pec_nodes] = True

    def edge_tail_head(self, t, k):
        """Local indices (a, b) of the tail and head nodes of local edge k of triangle t."""
        i, j = (k + 1) % 3, (k + 2) % 3
        return (i, j) if self.tris[t, i] < self.tris[t, j] else (j, i)


def _moment3(i, j, k):
    """Integral of lambda_i lambda_j lambda_k over a triangle divided by 2A.

    Uses int lambda_0^a lambda_1^b lambda_2^c dA = 2A a! b! c! / (a+b+c+2)!."""
    n = [0, 0, 0]
    for m in (i, j, k):
        n[m] += 1
    return math.factorial(n[0]) * math.factorial(n[1]) * math.factorial(n[2]) / math.factorial(5)


_M3 = np.array([[[_moment3(i, j, k) for k in range(3)] for j in range(3)] for i in range(3)])


def local_hodge_eps(mesh, eps0=1.0):
    """Local 3x3 matrices  eps0 * int_T rho W_k1 . W_k2  (App. B, defining integral).

    W_k = lambda_a grad(lambda_b) - lambda_b grad(lambda_a) for local edge k with tail a
    and head b; rho = sum_m rho_m lambda_m is exact for the linear element.  The
    integrand is a cubic in the barycentric coordinates, integrated exactly."""
    N2 = mesh.N2
    tails = np.zeros((N2, 3), np.int64)
    heads = np.zeros((N2, 3), np.int64)
    for k in range(3):
        i, j = (k + 1) % 3, (k + 2) % 3
        swap = mesh.tris[:, i] > mesh.tris[:, j]
        tails[:, k] = np.where(swap, j, i)
        heads[:, k] = np.where(swap, i, j)
    rho = mesh.nodes[mesh.tris][:, :, 1]
    G = np.einsum("tid,tjd->tij", mesh.grad, mesh.grad)       # grad(l_i) . grad(l_j)
    ar = np.arange(N2)
    T = np.zeros((N2, 3, 3))
    for k1 in range(3):
        a1, b1 = tails[:, k1], heads[:, k1]
        for k2 in range(3):
            a2, b2 = tails[:, k2], heads[:, k2]
            acc = np.zeros(N2)
            for m in range(3):
                acc += rho[:, m] * (G[ar, b1, b2] * _M3[a1, a2, m] - G[ar, b1, a2] * _M3[a1, b2, m]
                                    - G[ar, a1, b2] * _M3[b1, a2, m] + G[ar, a1, a2] * _M3[b1, b2, m])
            T[:, k1, k2] = eps0 * 2.0 * mesh.area * acc
    return T


def hodge_eps(mesh, eps0=1.0):
    """Global [star_eps] (N1 x N1, CSR), assembled from the local matrices."""
    T = local_hodge_eps(mesh, eps0)
    r = np.repeat(mesh.tri_edges, 3, axis=1).ravel()
    c = np.tile(mesh.tri_edges, (1, 3)).ravel()
    return sp.csr_matrix((T.ravel(), (r, c)), shape=(mesh.N1, mesh.N1))


def hodge_mu_inv(mesh, mu0=1.0):
    """Diagonal of [star_mu^-1]: (1/mu0) int_T rho W2.W2 with W2 = 1/A, i.e. rho_bar/(mu0 A)."""
    rho_bar = mesh.nodes[mesh.tris][:, :, 1].mean(1)
    return rho_bar / (mu0 * mesh.area)


def _edge_adjacency(mesh):
    """Boolean N1 x N1 matrix: edges sharing a triangle (diagonal included)."""
    Ti = sp.csr_matrix((np.ones(3 * mesh.N2), (np.repeat(np.arange(mesh.N2), 3),
                                                mesh.tri_edges.ravel())), shape=(mesh.N2, mesh.N1))
    A = (Ti.T @ Ti).tocsr()
    A.data[:] = 1.0
    return A


def spai_pattern(mesh, level):
    """Sparsity pattern S_j of column j: free edges within ``level`` triangle-hops of j."""
    adj = _edge_adjacency(mesh)
    P = sp.identity(mesh.N1, format="csr")
    for _ in range(level):
        P = (P @ adj).tocsr()
        P.data[:] = 1.0
    f = mesh.free
    return P[f][:, f].tocsc()


def spai(mesh, star_eps, level=2, drop_tol=1e-4):
    """Sparse approximate inverse M of [star_eps] restricted to the free edges.

    Column j minimises ||A m - e_j||_2 over vectors supported on the pattern S_j (a
    least-squares problem over the rows touched by S_j); entries below
    drop_tol * max|m| are dropped, then M <- (M + M^T)/2.  Returns M as CSR in the
    free-edge numbering."""
    f = mesh.free
    A = star_eps[f][:, f].tocsc()
    P = spai_pattern(mesh, level)
    n = len(f)
    rows, cols, vals = [], [], []
    for j in range(n):
        S = P.indices[P.indptr[j]:P.indptr[j + 1]]
        sub = A[:, S]
        R = np.unique(sub.indices)
        dense = sub[R].toarray()
        rhs = (R == j).astype(float)
        m, *_ = np.linalg.lstsq(dense, rhs, rcond=None)
        keep = np.abs(m) >= drop_tol * np.abs(m).max()
        rows.append(S[keep])
        cols.append(np.full(keep.sum(), j))
        vals.append(m[keep])
    M = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n))
    return (0.5 * (M + M.T)).tocsr()


def curl_curl(mesh, mu_inv):
    """K = D_curl^T [star_mu^-1] D_curl restricted to free edges."""
    Dc = mesh.Dcurl[:, mesh.free]
    return (Dc.T @ sp.diags(mu_inv) @ Dc).tocsr()


def power_start(n):
    """Deterministic start vector of the power iteration."""
    return 1.0 + 0.5 * np.sin(np.arange(1, n + 1, dtype=np.float64))


def dt_stable(mesh, M, mu_inv, iters=500):
    """Largest stable leapfrog step 2/sqrt(lambda_max(M K)) by power iteration.

    Eliminating B from Eqs. full_d_dfl / full_d_dal gives
    E^{n+1} - 2E^n + E^{n-1} = -dt^2 M K E^n, stable for dt^2 lambda_max < 4."""
    K = curl_curl(mesh, mu_inv)
    x = power_start(M.shape[0])
    x /= np.linalg.norm(x)
    lam = 0.0
    for _ in range(iters):
        y = M @ (K @ x)
        lam = np.linalg.norm(y)
        x = y / lam
    return 2.0 / math.sqrt(lam), lam


def field_energy(mesh, star_eps, mu_inv, E, B):
    """Per-radian field energy 1/2 E^T star_eps E + 1/2 B^T star_mu^-1 B."""
    return 0.5 * E @ (star_eps @ E) + 0.5 * np.sum(mu_inv * B * B)
