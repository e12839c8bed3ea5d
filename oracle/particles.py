"""ctypes wrapper of the plain-C FP64 particle step, and point location.  Test infrastructure."""
import ctypes
import os
import subprocess

import numpy as np
from scipy.spatial import cKDTree

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "particles.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lib = None

WALK_CAP = 16   # edge crossings per particle per step before it is dropped
BORIS, VAY = 0, 1   # velocity update of Eq. DLE (Sec. 3.3)


_LIB_OMP = os.path.join(_HERE, "_liboracle_omp.so")
_lib_omp = None


def build_oracle_lib(force=False):
    """Compile particles.c with gcc (no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def build_oracle_omp_lib(force=False):
    """The same source built with -fopenmp: the particle loop on all host cores with
    atomic accumulators.  Only the timed CPU baseline uses it; returns None when the
    compiler has no OpenMP."""
    if force or not os.path.exists(_LIB_OMP) or os.path.getmtime(_LIB_OMP) < os.path.getmtime(_SRC):
        tmp = _LIB_OMP + ".%d.tmp" % os.getpid()
        r = subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                            "-o", tmp, _SRC, "-lm"], capture_output=True)
        if r.returncode != 0:
            return None
        os.replace(tmp, _LIB_OMP)
    return _LIB_OMP


def _declare(lib):
    P = ctypes.c_void_p
    lib.oracle_push.argtypes = [P, P, P, P, P, P, P, P, P, ctypes.c_double,
                                ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                ctypes.c_int64, P, P, P, P, P, P, P]
    lib.oracle_kick.argtypes = [ctypes.c_int, ctypes.c_int64, P, P, P, ctypes.c_double,
                                ctypes.c_double, P]
    lib.oracle_deposit_charge.argtypes = [P, ctypes.c_int64, P, P, ctypes.c_double, P]
    lib.oracle_threads.argtypes = []
    return lib


def _load(threads=False):
    global _lib, _lib_omp
    if threads:
        if _lib_omp is None:
            path = build_oracle_omp_lib()
            if path is None:
                raise RuntimeError("gcc without OpenMP: no multi-threaded oracle build")
            _lib_omp = _declare(ctypes.CDLL(path))
        return _lib_omp
    if _lib is None:
        _lib = _declare(ctypes.CDLL(build_oracle_lib()))
    return _lib


def host_threads(threads=False):
    """Host threads the particle loop of the plain (1) or the OpenMP build runs on."""
    return int(_load(threads).oracle_threads())


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class PushMesh:
    """Contiguous int32/float64 copies of the mesh arrays the C step reads."""

    def __init__(self, mesh):
        self.tri_nodes = np.ascontiguousarray(mesh.tris, np.int32)
        self.tri_edges = np.ascontiguousarray(mesh.tri_edges, np.int32)
        self.tri_nbr = np.ascontiguousarray(mesh.nbr, np.int32)
        self.tri_btag = np.ascontiguousarray(mesh.tri_btag, np.int32)
        self.node_zr = np.ascontiguousarray(mesh.nodes, np.float64)
        self.grad = np.ascontiguousarray(mesh.grad, np.float64)
        self.area = np.ascontiguousarray(mesh.area, np.float64)


def kick(pusher, u, Ef, Bf, h, c):
    """The velocity update of Eq. DLE alone (BORIS or VAY) for rows of u, E and B in local
    (rho, phi, z) components; h = q dt / (2 m)."""
    lib = _load()
    u = np.ascontiguousarray(np.atleast_2d(u), np.float64)
    Ef = np.ascontiguousarray(np.broadcast_to(Ef, u.shape), np.float64)
    Bf = np.ascontiguousarray(np.broadcast_to(Bf, u.shape), np.float64)
    out = np.zeros_like(u)
    lib.oracle_kick(int(pusher), len(u), _ptr(u), _ptr(Ef), _ptr(Bf), float(h), float(c),
                    _ptr(out))
    return out


def push(pm, E, Bavg, bz, dt, qm, c, q_src, tri, lam, u, J, Q, Qabs, max_cross=WALK_CAP,
         pusher=BORIS, threads=False):
    """One particle step in place (see oracle_push in particles.c).  Returns counters
    (absorbed, walk-cap overflows, edge crossings).  threads=True runs the OpenMP build
    (all host cores, atomic sums; the timed CPU baseline only)."""
    lib = _load(threads)
    for a, dt_ in ((tri, np.int32), (lam, np.float64), (u, np.float64), (J, np.float64),
                   (Q, np.float64), (Qabs, np.float64)):
        assert a.dtype == dt_ and a.flags.c_contiguous
    E = np.ascontiguousarray(E, np.float64)
    Bavg = np.ascontiguousarray(Bavg, np.float64)
    cnt = np.zeros(3, np.int64)
    lib.oracle_push(_ptr(pm.tri_nodes), _ptr(pm.tri_edges), _ptr(pm.tri_nbr), _ptr(pm.tri_btag),
                    _ptr(pm.node_zr), _ptr(pm.grad), _ptr(pm.area), _ptr(E), _ptr(Bavg),
                    float(bz), float(dt), float(qm), float(c), float(q_src), int(max_cross),
                    int(pusher), int(len(tri)), _ptr(tri), _ptr(lam), _ptr(u), _ptr(J), _ptr(Q), _ptr(Qabs),
                    _ptr(cnt))
    return cnt


def deposit_charge(pm, tri, lam, q_src, Q):
    """Eq. charge for all live particles, added into Q."""
    lib = _load()
    lib.oracle_deposit_charge(_ptr(pm.tri_nodes), int(len(tri)), _ptr(tri), _ptr(lam),
                              float(q_src), _ptr(Q))


def barycentric(mesh, t, z, rho):
    """lambda_k(p) = signed area of (p, p_{k+1}, p_{k+2}) / area of the triangle."""
    p = mesh.nodes[mesh.tris[t]]
    lam = np.zeros((len(t), 3))
    for k in range(3):
        a, b = (k + 1) % 3, (k + 2) % 3
        lam[:, k] = ((p[:, a, 0] - z) * (p[:, b, 1] - rho)
                     - (p[:, b, 0] - z) * (p[:, a, 1] - rho)) / (2.0 * mesh.area[t])
    return lam


def locate(mesh, z, rho, k_near=16):
    """Containing triangle of each point: among the k_near triangles with the nearest
    centroids, the one whose smallest barycentric coordinate is largest (ties: lower
    triangle index); falls back to all triangles.  Returns (tri, lambda); tri = -1 for
    points outside the mesh."""
    z = np.asarray(z, float)
    rho = np.asarray(rho, float)
    cen = mesh.nodes[mesh.tris].mean(1)
    k = min(k_near, mesh.N2)
    _, cand = cKDTree(cen).query(np.stack([z, rho], 1), k=k)
    cand = np.asarray(cand).reshape(len(z), k)
    best_t = -np.ones(len(z), np.int64)
    best_m = np.full(len(z), -np.inf)
    for j in range(k):
        t = cand[:, j]
        mn = barycentric(mesh, t, z, rho).min(1)
        better = (mn > best_m) | ((mn == best_m) & (t < best_t))
        best_t = np.where(better, t, best_t)
        best_m = np.where(better, mn, best_m)
    miss = best_m < -1e-12
    for p in np.flatnonzero(miss):
        allt = np.arange(mesh.N2)
        mn = barycentric(mesh, allt, np.full(mesh.N2, z[p]), np.full(mesh.N2, rho[p])).min(1)
        best_t[p] = int(np.argmax(mn))
        best_m[p] = mn[best_t[p]]
    tri = np.where(best_m >= -1e-12, best_t, -1).astype(np.int32)
    lam = np.zeros((len(z), 3))
    ok = tri >= 0
    lam[ok] = barycentric(mesh, tri[ok].astype(np.int64), z[ok], rho[ok])
    return tri, lam
