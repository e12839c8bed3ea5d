"""Batching of independent simulations by mesh union (host side, numpy only).

Several meridian-plane meshes, each with its particles, are placed side by side along z
(each shifted past the previous ones plus a gap) and handed to the library as one mesh
and one particle set.  Every operator of the method is local to a mesh (edge orientation
and numbering follow the node numbering, the SPAI pattern grows from neighbouring edges,
the particle walk never leaves a mesh), so the union's operators are block-diagonal and
one simulation advances all instances; the common time step must respect the smallest
instance limit, which the union's stable step is.
"""
import numpy as np

GAP = 1e-2   # z gap between consecutive meshes (SI metres)


def union(instances, gap=GAP):
    """One mesh and one particle set holding all instances.

    Each instance is a dict with nodes (n x 2: z, rho), tris, be, bt (boundary edges and
    tags) and particles z, r, ur, up, uz.  Returns the union arrays and, per instance, the
    offsets of its nodes, triangles and particles (``node_off``, ``tri_off``, ``part_off``,
    length len(instances) + 1) and its z shift (``shift``)."""
    nodes, tris, be, bt, zs, rs, urs, ups, uzs = [], [], [], [], [], [], [], [], []
    node_off, tri_off, part_off, shift = [0], [0], [0], []
    z0 = 0.0
    for ins in instances:
        lo, hi = float(ins["nodes"][:, 0].min()), float(ins["nodes"][:, 0].max())
        dz = z0 - lo
        nn = ins["nodes"].copy()
        nn[:, 0] += dz
        nodes.append(nn)
        tris.append(ins["tris"] + node_off[-1])
        be.append(ins["be"] + node_off[-1])
        bt.append(ins["bt"])
        zs.append(ins["z"] + dz)
        rs.append(ins["r"])
        urs.append(ins["ur"])
        ups.append(ins["up"])
        uzs.append(ins["uz"])
        shift.append(dz)
        node_off.append(node_off[-1] + len(ins["nodes"]))
        tri_off.append(tri_off[-1] + len(ins["tris"]))
        part_off.append(part_off[-1] + len(ins["z"]))
        z0 += (hi - lo) + gap
    cat = np.concatenate
    return dict(nodes=cat(nodes), tris=cat(tris).astype(np.int32),
                be=cat(be).astype(np.int32), bt=cat(bt).astype(np.int32),
                z=cat(zs), r=cat(rs), ur=cat(urs), up=cat(ups), uz=cat(uzs),
                node_off=np.array(node_off), tri_off=np.array(tri_off),
                part_off=np.array(part_off), shift=np.array(shift))


def partition(work, n_ranks):
    """Instances to ranks for a sweep sharded across GPUs (one union per rank, no data
    exchanged): longest work first, each to the least-loaded rank (ties: the lower rank),
    so the slowest rank carries at most 4/3 of the optimum.  ``work`` is a per-instance cost
    (e.g. particles + triangles).  Returns one ascending list of instance indices per rank."""
    work = np.asarray(work, float)
    loads = np.zeros(n_ranks)
    parts = [[] for _ in range(n_ranks)]
    for i in sorted(range(len(work)), key=lambda k: (-work[k], k)):
        r = int(np.argmin(loads))
        parts[r].append(i)
        loads[r] += work[i]
    return [sorted(p) for p in parts]
