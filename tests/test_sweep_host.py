"""Batched ripple sweep, host side: the 64 instance parameters stay in their ranges, and
the union of instances is one valid mesh whose counts are the instances' sums and whose
stable step is the smallest instance's (its operators are block-diagonal)."""
import numpy as np
import pytest

from workloads.sweep import sweep_params, sweep_instance, union
from workloads.bwo import EPS0, MU0, C0


@pytest.fixture(scope="module")
def pic():
    import paper_1701_03784_gb300 as pkg
    pkg.build()
    from paper_1701_03784_gb300 import pic as p
    return p


def test_parameters_in_range():
    for i in range(64):
        p = sweep_params(i)
        assert 0.2e-2 <= p["depth"] <= 0.6e-2 and 1.4e-2 <= p["period"] <= 2.0e-2
        assert 8 <= p["n_periods"] <= 16 and 300e3 <= p["voltage"] <= 500e3
        assert 1e3 <= p["current"] <= 5e3 and 20_000 <= p["n_tri"] <= 80_000


def test_union_is_the_instances_side_by_side(pic):
    ins = [sweep_instance(i, scale=1e-4) for i in (0, 27, 5)]   # 27 needs a finer wall
    u = union(ins)
    mk = lambda x: pic.pic_mesh_create(x["nodes"], x["tris"], x["be"], x["bt"], eps0=EPS0,
                                       mu0=MU0, c=C0, precision=pic.PIC_FP32)
    mu = mk(u)
    info = pic.pic_mesh_info(mu)
    parts = [pic.pic_mesh_info(mk(x)) for x in ins]
    for k in ("n_nodes", "n_edges", "n_tris", "n_free_edges"):
        assert info[k] == sum(p[k] for p in parts), k
    # the union's mesh of instance i is instance i's, shifted
    assert np.all(np.diff(u["shift"]) > 0)
    for i, x in enumerate(ins):
        a, b = u["node_off"][i], u["node_off"][i + 1]
        assert np.allclose(u["nodes"][a:b, 0] - u["shift"][i], x["nodes"][:, 0], atol=1e-15)
        assert np.array_equal(u["nodes"][a:b, 1], x["nodes"][:, 1])
    dts = [pic.pic_spai_build(mk(x), 2, 1e-4) for x in ins]
    dtu = pic.pic_spai_build(mu, 2, 1e-4)
    assert abs(dtu - min(dts)) <= 1e-3 * min(dts)


def test_partition_of_instances_over_ranks():
    """Every instance on exactly one rank, ascending lists, and the greedy longest-first
    bound: no rank above 4/3 of the best possible makespan's lower bound (the larger of
    the mean load and the largest instance)."""
    from paper_1701_03784_gb300.batch import partition
    from workloads.sweep import sweep_params, sweep_particles
    work = [sweep_particles(i) + sweep_params(i)["n_tri"] for i in range(64)]
    for n in (1, 2, 3, 8):
        parts = partition(work, n)
        assert len(parts) == n
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(64))
        assert all(p == sorted(p) for p in parts)
        loads = [sum(work[i] for i in p) for p in parts]
        bound = max(sum(work) / n, max(work))
        assert max(loads) <= 4.0 / 3.0 * bound
    assert partition(work, 2) == partition(work, 2)
    assert partition([5.0, 1.0, 1.0], 4) == [[0], [1], [2], []]
