"""Seeded jittered-point Delaunay meshes of axisymmetric domains in the meridian plane.

A domain is {(z, rho): z0 <= z <= z1, 0 <= rho <= R(z)}.  Boundary points are laid on
the axis, both end planes and the wall curve at the target spacing; interior points
are a jittered triangular lattice kept clear of the boundary.  scipy's Delaunay
triangulation of the point set is clipped to the domain by triangle centroid.
"""
import numpy as np
from scipy.spatial import Delaunay, cKDTree

from . import BC_PEC, BC_AXIS, BC_ABSORB


def _wall_points(R, z0, z1, h, breaks=()):
    """Points on rho = R(z) at arc-length spacing close to h, endpoints included.

    Each piece between consecutive break points (slope discontinuities of the wall) is
    sampled separately so that every break point is a mesh node."""
    knots = [z0] + sorted(b for b in breaks if z0 < b < z1) + [z1]
    out = []
    for a, b in zip(knots[:-1], knots[1:]):
        zz = np.linspace(a, b, 100001)
        rr = R(zz)
        s = np.concatenate([[0.0], np.cumsum(np.hypot(np.diff(zz), np.diff(rr)))])
        n = max(1, int(round(s[-1] / h)))
        st = np.linspace(0.0, s[-1], n + 1)
        zw = np.interp(st, s, zz)
        zw[0], zw[-1] = a, b
        out.append(zw if not out else zw[1:])
    zw = np.concatenate(out)
    return zw, R(zw)


def _segment_points(a, b, h):
    n = max(1, int(round(abs(b - a) / h)))
    return np.linspace(a, b, n + 1)


def _polyline_points(corners, h):
    """Points along a polyline (corners included) at spacing close to h per segment."""
    out = [corners[:1]]
    for a, b in zip(corners[:-1], corners[1:]):
        n = max(1, int(round(np.hypot(*(b - a)) / h)))
        t = np.linspace(0.0, 1.0, n + 1)[1:, None]
        out.append(a + t * (b - a))
    return np.concatenate(out, 0)


def jittered_delaunay(z0, z1, R, n_tri, seed, jitter=0.2,
                      end_tags=(BC_PEC, BC_PEC), wall_tag=BC_PEC, breaks=(), wall_refine=1.0,
                      wall_corners=None):
    """Mesh of {z0<=z<=z1, 0<=rho<=R(z)} with about ``n_tri`` triangles.

    ``wall_refine`` < 1 places the wall points closer than the interior spacing (for
    walls whose curvature a coarse mesh does not resolve).  ``wall_corners`` (an array of
    (z, rho) corners from (z0, R(z0)) to (z1, R(z1))) lays the wall on that polyline
    instead of sampling the curve, e.g. a staircase with vertical steps (R must then give
    the larger radius exactly at a step).
    Returns (nodes, tris, bedges, btags); see the package docstring for layouts.
    """
    rng = np.random.default_rng(seed)
    zz = np.linspace(z0, z1, 20001)
    rz = R(zz)
    area = float(np.sum(0.5 * (rz[1:] + rz[:-1]) * np.diff(zz)))
    # equilateral lattice: one triangle per sqrt(3)/4 h^2 of area
    h = np.sqrt(4.0 * area / (np.sqrt(3.0) * n_tri))

    pts = []
    # axis rho = 0 (corners included)
    za = _segment_points(z0, z1, h)
    pts.append(np.stack([za, np.zeros_like(za)], 1))
    # end planes (rho > 0 part; top corners included)
    for ze in (z0, z1):
        re = _segment_points(0.0, float(R(np.array([ze]))[0]), h)[1:]
        pts.append(np.stack([np.full_like(re, ze), re], 1))
    # wall (corners excluded: they belong to the end planes)
    if wall_corners is None:
        zw, rw = _wall_points(R, z0, z1, h * wall_refine, breaks)
        pts.append(np.stack([zw[1:-1], rw[1:-1]], 1))
    else:
        pts.append(_polyline_points(np.asarray(wall_corners, float), h * wall_refine)[1:-1])
    n_boundary = sum(len(p) for p in pts)

    # interior jittered triangular lattice
    dy = h * np.sqrt(3.0) / 2.0
    rmax = float(rz.max())
    rows = np.arange(1, int(rmax / dy) + 2)
    gz, gr = [], []
    for j in rows:
        zs = z0 + (np.arange(-1, int((z1 - z0) / h) + 2) + 0.5 * (j % 2)) * h
        gz.append(zs)
        gr.append(np.full_like(zs, j * dy))
    gz = np.concatenate(gz)
    gr = np.concatenate(gr)
    gz = gz + rng.uniform(-jitter, jitter, gz.shape) * h
    gr = gr + rng.uniform(-jitter, jitter, gr.shape) * h
    margin = 0.6 * h
    keep = ((gz > z0 + margin) & (gz < z1 - margin) & (gr > margin)
            & (gr < R(np.clip(gz, z0, z1)) - margin * 0.5))
    # distance to the wall measured along the normal (dense wall sampling)
    if wall_corners is None:
        zd = np.linspace(z0, z1, int(40 * (z1 - z0) / h) + 2)
        dense = np.stack([zd, R(zd)], 1)
    else:
        dense = _polyline_points(np.asarray(wall_corners, float), h / 40.0)
    dist, _ = cKDTree(dense).query(np.stack([gz, gr], 1))
    keep &= dist > margin
    pts.append(np.stack([gz[keep], gr[keep]], 1))
    P = np.concatenate(pts, 0)

    tri = Delaunay(P).simplices.astype(np.int64)
    # keep a triangle when its centroid is inside and none of its edge midpoints lies
    # outside the wall by more than a chord's sagitta (rejects hull triangles that
    # bridge the valleys of a rippled wall)
    c = P[tri].mean(1)
    inside = c[:, 1] < R(np.clip(c[:, 0], z0, z1))
    for i, j in ((0, 1), (1, 2), (2, 0)):
        mid = 0.5 * (P[tri[:, i]] + P[tri[:, j]])
        inside &= mid[:, 1] <= R(np.clip(mid[:, 0], z0, z1)) + 0.05 * h
    tri = tri[inside]
    a = P[tri]
    sarea = 0.5 * ((a[:, 1, 0] - a[:, 0, 0]) * (a[:, 2, 1] - a[:, 0, 1])
                   - (a[:, 2, 0] - a[:, 0, 0]) * (a[:, 1, 1] - a[:, 0, 1]))
    good = np.abs(sarea) > 1e-6 * h * h
    tri, sarea = tri[good], sarea[good]
    neg = sarea < 0
    tri[neg] = tri[neg][:, [0, 2, 1]]

    # drop unreferenced points, renumber
    used = np.zeros(len(P), bool)
    used[tri.ravel()] = True
    remap = -np.ones(len(P), np.int64)
    remap[used] = np.arange(used.sum())
    nodes = P[used]
    tris = remap[tri]

    bedges, btags = _boundary_edges(nodes, tris, z0, z1, end_tags, wall_tag)
    # every boundary edge must join two boundary points: the Delaunay conformed
    is_bpt = np.zeros(len(P), bool)
    is_bpt[:n_boundary] = True
    bpt = is_bpt[used]
    if not np.all(bpt[bedges]):
        raise RuntimeError("jittered_delaunay: triangulation does not conform to the boundary")
    # one boundary loop without pinch points: every boundary node has two boundary edges
    deg = np.bincount(bedges.ravel(), minlength=len(nodes))
    n_edges = len(bedges) + (3 * len(tris) - len(bedges)) // 2
    if np.any((deg != 0) & (deg != 2)) or len(nodes) - n_edges + len(tris) != 1:
        raise RuntimeError("jittered_delaunay: mesh is not a disk")
    return nodes.astype(np.float64), tris.astype(np.int32), bedges, btags


def _boundary_edges(nodes, tris, z0, z1, end_tags, wall_tag):
    e = np.concatenate([tris[:, [1, 2]], tris[:, [2, 0]], tris[:, [0, 1]]], 0)
    e = np.sort(e, 1)
    key = e[:, 0] * (len(nodes) + 1) + e[:, 1]
    uk, cnt = np.unique(key, return_counts=True)
    bk = uk[cnt == 1]
    be = np.stack([bk // (len(nodes) + 1), bk % (len(nodes) + 1)], 1)
    zr = nodes[be]
    tags = np.full(len(be), wall_tag, np.int32)
    tags[(zr[:, 0, 0] == z0) & (zr[:, 1, 0] == z0)] = end_tags[0]
    tags[(zr[:, 0, 0] == z1) & (zr[:, 1, 0] == z1)] = end_tags[1]
    tags[(zr[:, 0, 1] == 0.0) & (zr[:, 1, 1] == 0.0)] = BC_AXIS
    return be.astype(np.int32), tags


def rect_mesh(Lz, a, n_tri, seed, end_tags=(BC_PEC, BC_PEC), wall_tag=BC_PEC, z0=0.0):
    """Jittered mesh of the rectangle [z0, z0+Lz] x [0, a]."""
    return jittered_delaunay(z0, z0 + Lz, lambda z: np.full_like(np.asarray(z, float), a),
                             n_tri, seed, end_tags=end_tags, wall_tag=wall_tag)


def cavity_mesh(a=0.5, L=1.0, n_tri=2000, seed=1000):
    """Closed PEC cylindrical cavity, radius a and length L (normalised units)."""
    return rect_mesh(L, a, n_tri, seed)


def bwo_wall(r0=1.5e-2, ripple=0.4e-2, period=1.67e-2, n_periods=12, guide=3e-2):
    """Wall radius R(z) of the rippled slow-wave structure with straight guide sections.

    R(z) = r0 + ripple * sin(2 pi (z - guide) / period) over the ripple section, r0 in
    the input/output guides.  Returns (R, z_end, (z_sws_start, z_sws_end)).
    """
    zs0 = guide
    zs1 = guide + n_periods * period
    z_end = zs1 + guide

    def R(z):
        z = np.asarray(z, float)
        inside = (z > zs0) & (z < zs1)
        return np.where(inside, r0 + ripple * np.sin(2 * np.pi * (z - zs0) / period), r0)

    return R, z_end, (zs0, zs1)


def bwo_mesh(n_tri=200_000, seed=1002, wall_refine=1.0, **wall):
    """Single backward-wave oscillator: rippled wall, 12 periods, guides, SI metres."""
    R, z_end, sws = bwo_wall(**wall)
    return jittered_delaunay(0.0, z_end, R, n_tri, seed,
                             end_tags=(BC_ABSORB, BC_ABSORB), wall_tag=BC_PEC, breaks=sws,
                             wall_refine=wall_refine)


def bwo_small_mesh(n_tri=3000, seed=1012):
    """Two-period rippled section with 0.5 cm guides: a BWO-shaped mesh small enough for
    the oracle to step in seconds."""
    return bwo_mesh(n_tri=n_tri, seed=seed, n_periods=2, guide=0.5e-2)


def diode_mesh(n_tri=20_000, seed=1001, gap=1e-2, radius=2e-2, grade=1.0):
    """Planar diode: cathode plane z=0, anode plane z=gap, outer wall at rho=radius.

    grade < 1 compresses the cells toward the cathode: node z -> gap (g s + (1 - g) s^2),
    s = z / gap, a monotone map that keeps rho, the two planes and the triangles'
    orientation; the first cells are g times as deep (the space-charge-limited potential
    varies as z^(4/3) there) and the last ones 2 - g times."""
    nodes, tris, be, bt = rect_mesh(gap, radius, n_tri, seed)
    if grade != 1.0:
        s = nodes[:, 0] / gap
        z = gap * (grade * s + (1.0 - grade) * s * s)
        z[nodes[:, 0] == 0.0] = 0.0
        z[nodes[:, 0] == gap] = gap
        nodes = np.stack([z, nodes[:, 1]], 1)
    return nodes, tris, be, bt


def sws_cell_mesh(n_tri, seed=1020, staircase=False, r0=15.0e-3, ripple=2.1e-3,
                  period=7.5e-3):
    """One period of a rippled slow-wave structure between two ripple maxima,
    R(z) = r0 + ripple cos(2 pi z / period) for z in [0, period], conducting end planes
    (the symmetry planes: the cell's TM01 resonances are the 0 and pi points of the
    periodic structure's dispersion).  staircase=True replaces the wall by steps of the
    mesh spacing h in both z and rho (each z-bin at R of its centre rounded to h): the
    boundary a structured mesh of that spacing would see."""
    def R(z):
        return r0 + ripple * np.cos(2.0 * np.pi * np.asarray(z, float) / period)

    if not staircase:
        for refine in (0.7, 0.5, 0.35, 0.25):
            try:
                return jittered_delaunay(0.0, period, R, n_tri, seed, wall_refine=refine)
            except RuntimeError:
                continue
        raise RuntimeError("sws_cell_mesh: no conforming mesh")
    zz = np.linspace(0.0, period, 20001)
    area = float(np.sum(0.5 * (R(zz)[1:] + R(zz)[:-1]) * np.diff(zz)))
    h = np.sqrt(4.0 * area / (np.sqrt(3.0) * n_tri))
    nb = max(2, int(round(period / h)))
    edges = np.linspace(0.0, period, nb + 1)
    level = np.maximum(np.round(R(0.5 * (edges[:-1] + edges[1:])) / h), 1.0) * h
    corners = [(0.0, level[0])]
    for k in range(nb):
        corners.append((edges[k + 1], level[k]))
        if k + 1 < nb and level[k + 1] != level[k]:
            corners.append((edges[k + 1], level[k + 1]))

    def Rs(z):
        z = np.asarray(z, float)
        k = np.clip(np.searchsorted(edges, z, side="right") - 1, 0, nb - 1)
        r = level[k]
        # at a step the larger of the two radii (the step's edge belongs to the domain)
        at = np.isclose(z, edges[np.clip(k, 0, nb)]) & (k > 0)
        return np.where(at, np.maximum(r, level[np.maximum(k - 1, 0)]), r)

    return jittered_delaunay(0.0, period, Rs, n_tri, seed, wall_refine=0.7,
                             wall_corners=np.array(corners))


def two_triangle_mesh():
    """Unit square [0,1]x[0.5,1.5] split along a diagonal; off-axis, all PEC."""
    nodes = np.array([[0.0, 0.5], [1.0, 0.5], [1.0, 1.5], [0.0, 1.5]])
    tris = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    bedges = np.array([[0, 1], [1, 2], [2, 3], [0, 3]], np.int32)
    return nodes, tris, bedges, np.full(4, BC_PEC, np.int32)


def four_triangle_mesh():
    """Square [0,2]x[0,2] around a centre node, touching the axis rho=0 on one side."""
    nodes = np.array([[0.0, 0.0], [2.0, 0.0], [2.0, 2.0], [0.0, 2.0], [1.0, 0.9]])
    tris = np.array([[0, 1, 4], [1, 2, 4], [2, 3, 4], [3, 0, 4]], np.int32)
    bedges = np.array([[0, 1], [1, 2], [2, 3], [0, 3]], np.int32)
    btags = np.array([BC_AXIS, BC_PEC, BC_PEC, BC_PEC], np.int32)
    return nodes, tris, bedges, btags
