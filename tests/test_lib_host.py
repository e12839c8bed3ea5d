"""The C-ABI library on the CPU: it loads, exports every function include/pic.h declares,
rejects bad meshes, and its host-side setup (edge numbering, SPAI, stable step) matches
the oracle.  No GPU needed: these calls do not touch the device."""
import os
import re
import subprocess
import sys

import numpy as np
import pytest

import workloads as W
from oracle.operators import Mesh, hodge_eps, hodge_mu_inv, spai, dt_stable

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pic():
    import paper_1701_03784_gb300 as pkg
    pkg.build()
    from paper_1701_03784_gb300 import pic as p
    return p


def _declared():
    src = open(os.path.join(ROOT, "include", "pic.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pic_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(pic):
    names = _declared()
    assert len(names) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", pic.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    assert set(pic.EXPORTED) <= set(names)


def test_bad_meshes_are_rejected(pic):
    nodes, tris, be, bt = W.two_triangle_mesh()
    with pytest.raises(pic.PicError) as e:
        pic.pic_mesh_create(nodes, np.array([[0, 1, 1], [0, 2, 3]]), be, bt)
    assert e.value.status == pic.PIC_ERR_MESH
    with pytest.raises(pic.PicError) as e:
        pic.pic_mesh_create(nodes, tris, be[:3], bt[:3])          # a boundary edge untagged
    assert e.value.status == pic.PIC_ERR_MESH
    with pytest.raises(pic.PicError) as e:
        pic.pic_mesh_create(nodes, np.array([[0, 1, 9], [0, 2, 3]]), be, bt)
    assert e.value.status == pic.PIC_ERR_ARG
    bad = nodes.copy()
    bad[0, 1] = -0.1
    with pytest.raises(pic.PicError) as e:
        pic.pic_mesh_create(bad, tris, be, bt)
    assert e.value.status == pic.PIC_ERR_ARG
    with pytest.raises(pic.PicError) as e:
        pic.pic_mesh_create(nodes, tris, np.vstack([be, [[0, 2]]]), np.append(bt, 1))
    assert e.value.status == pic.PIC_ERR_MESH                     # interior edge listed
    folded = np.vstack([nodes, [[0.6, 0.8]]])                     # both triangles below 0-2
    with pytest.raises(pic.PicError) as e:
        pic.pic_mesh_create(folded, np.array([[0, 1, 2], [0, 4, 2]]),
                            np.array([[0, 1], [1, 2], [0, 4], [4, 2]]), np.ones(4, np.int32))
    assert e.value.status == pic.PIC_ERR_MESH and "overlap" in pic.pic_last_error()
    with pytest.raises(pic.PicError) as e:
        pic.pic_mesh_create(nodes, tris, be, bt, walk_cap=4097)     # unbounded walks
    assert e.value.status == pic.PIC_ERR_ARG
    m = pic.pic_mesh_create(nodes, tris, be, bt)
    with pytest.raises(pic.PicError) as e:
        pic.pic_sim_create(m, 0.01)                               # no SPAI yet
    assert e.value.status == pic.PIC_ERR_STATE
    assert "pic_sim_create" in pic.pic_last_error()


@pytest.mark.parametrize("which", ["cavity", "bwo_small", "four"])
def test_host_setup_matches_oracle(pic, which):
    mk = {"cavity": lambda: W.cavity_mesh(n_tri=600, seed=3),
          "bwo_small": lambda: W.bwo_small_mesh(n_tri=3000, seed=4),
          "four": W.four_triangle_mesh}[which]
    nodes, tris, be, bt = mk()
    eps0, mu0 = (8.8541878128e-12, 1.25663706212e-6) if which == "bwo_small" else (1.0, 1.0)
    om = Mesh(nodes, tris, be, bt)
    m = pic.pic_mesh_create(nodes, tris, be, bt, eps0=eps0, mu0=mu0)
    info = pic.pic_mesh_info(m)
    assert (info["n_nodes"], info["n_edges"], info["n_tris"]) == (om.N0, om.N1, om.N2)
    assert np.array_equal(pic.pic_mesh_edges(m), om.edge_nodes)
    assert info["n_free_edges"] == len(om.free)
    level = 2 if which != "four" else 6
    dt = pic.pic_spai_build(m, level, 1e-4 if which != "four" else 0.0)
    fe, ip, ix, vv = pic.pic_spai_get(m)
    assert np.array_equal(fe, om.free)
    A = hodge_eps(om, eps0)
    M = spai(om, A, level, 1e-4 if which != "four" else 0.0).tocsr()
    M.sort_indices()
    assert np.array_equal(ip, M.indptr) and np.array_equal(ix, M.indices)
    assert np.allclose(vv, M.data, rtol=1e-9, atol=1e-12 * np.abs(M.data).max())
    dt_o, _ = dt_stable(om, M, hodge_mu_inv(om, mu0))
    assert abs(dt - dt_o) <= 1e-9 * dt_o


def test_header_is_plain_c():
    """include/pic.h compiles as C99 (the boundary takes plain pointers and sizes only)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    hdr = os.path.join(os.path.dirname(__file__), "..", "include", "pic.h")
    r = subprocess.run([gcc, "-std=c99", "-fsyntax-only", "-Wall", "-Werror", "-x", "c", hdr],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


_OOM_CHILD = r'''
import resource, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_1701_03784_gb300 import pic as P

n = 600                                  # structured grid: 720k triangles
z, r = np.meshgrid(np.linspace(0, 1, n + 1), np.linspace(0, 1, n + 1), indexing="ij")
nodes = np.stack([z.ravel(), r.ravel()], 1)
idx = lambda i, j: i * (n + 1) + j
i, j = [a.ravel() for a in np.meshgrid(np.arange(n), np.arange(n), indexing="ij")]
tris = np.concatenate([np.stack([idx(i, j), idx(i + 1, j), idx(i + 1, j + 1)], 1),
                       np.stack([idx(i, j), idx(i + 1, j + 1), idx(i, j + 1)], 1)])
k = np.arange(n)
be = np.concatenate([np.stack([idx(k, 0), idx(k + 1, 0)], 1), np.stack([idx(k, n), idx(k + 1, n)], 1),
                     np.stack([idx(0, k), idx(0, k + 1)], 1), np.stack([idx(n, k), idx(n, k + 1)], 1)])
bt = np.concatenate([np.full(n, P.PIC_BC_AXIS), np.full(3 * n, P.PIC_BC_PEC)])
# in the binding's types already, so that only the library allocates under the cap
nodes, tris = np.ascontiguousarray(nodes, np.float64), np.ascontiguousarray(tris, np.int32)
be, bt = np.ascontiguousarray(be, np.int32), np.ascontiguousarray(bt, np.int32)
vm = int([l for l in open("/proc/self/status") if l.startswith("VmSize")][0].split()[1])
resource.setrlimit(resource.RLIMIT_AS, (vm * 1024 + 32 * 2 ** 20, resource.RLIM_INFINITY))
try:
    P.pic_mesh_create(nodes, tris, be, bt)
    print("created")
except P.PicError as e:
    print("status:", e)
'''


def test_host_allocation_failure_returns_a_status(pic, tmp_path):
    """Every call returns a status and never aborts: with the address space capped just
    above what the process holds, building a 720k-triangle mesh runs out of host memory
    inside the library, and the call reports PIC_ERR_OOM instead of ending the process."""
    script = tmp_path / "oom_child.py"
    script.write_text(_OOM_CHILD)
    out = subprocess.run([sys.executable, str(script), ROOT], capture_output=True, text=True,
                         timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    assert "PIC_ERR_OOM" in out.stdout and "out of host memory" in out.stdout, out.stdout


def test_host_faults_are_statuses(pic):
    """Faults injected on the host come back as statuses before any device work: a time
    step above the SPAI-stable limit (PIC_ERR_UNSTABLE), non-finite or non-positive steps
    and bad sizes (PIC_ERR_ARG), and SPAI parameters out of range."""
    nodes, tris, be, bt = W.cavity_mesh(n_tri=300, seed=3)
    m = pic.pic_mesh_create(nodes, tris, be, bt)
    for level, tol in ((-1, 1e-4), (9, 1e-4), (2, -1e-4), (2, float("nan")), (2, 1.0)):
        with pytest.raises(pic.PicError) as e:
            pic.pic_spai_build(m, level, tol)
        assert e.value.status == pic.PIC_ERR_ARG
    dt = pic.pic_spai_build(m, 2, 1e-4)
    for bad_dt in (1.01 * dt, float("inf")):
        with pytest.raises(pic.PicError) as e:
            pic.pic_sim_create(m, bad_dt, torch_memory=False)
        assert e.value.status == pic.PIC_ERR_UNSTABLE and "stable" in pic.pic_last_error()
    for args in ((0.0, 0.0, 10), (-dt, 0.0, 10), (float("nan"), 0.0, 10),
                 (0.5 * dt, float("inf"), 10), (0.5 * dt, float("nan"), 10),
                 (0.5 * dt, 0.0, -1), (0.5 * dt, 0.0, 1 << 31)):
        with pytest.raises(pic.PicError) as e:
            pic.pic_sim_create(m, args[0], args[1], args[2], torch_memory=False)
        assert e.value.status == pic.PIC_ERR_ARG


def test_binding_fails_loudly_without_the_library(tmp_path):
    """No fallback: a copy of the Python package without the built library refuses to
    import its binding."""
    import shutil
    pkg = tmp_path / "paper_1701_03784_gb300"
    pkg.mkdir()
    src = os.path.join(ROOT, "paper_1701_03784_gb300")
    for f in os.listdir(src):
        if f.endswith(".py"):
            shutil.copy(os.path.join(src, f), pkg / f)
    code = ("import sys; sys.path.insert(0, %r)\n"
            "try:\n    import paper_1701_03784_gb300.pic\nexcept ImportError as e:\n"
            "    print('refused:', e)\n" % str(tmp_path))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                         timeout=120, cwd=str(tmp_path))
    assert out.returncode == 0 and "refused: libpic_gb300.so is not built" in out.stdout, out


def test_handles_keep_the_allocator_hooks_they_were_made_with(pic):
    """The library calls a handle's allocator hooks again when the handle is freed, so the
    binding keeps their ctypes trampolines alive with the handle, even after the process
    installs other hooks."""
    import gc
    pic.pic_set_allocator(lambda n, ctx: None, lambda p, ctx: None)
    hooks = pic._torch_hooks
    s = pic.Sim(None, None)
    n = pic.Mlp(None, 1, [1, 1])
    pic.pic_set_allocator()
    gc.collect()
    assert pic._torch_hooks is None
    assert s._hooks is hooks and n._hooks is hooks and hooks is not None
    # both kinds of handle are freed at exit, while the hooks' owner is still alive
    assert s in pic._live_sims and n in pic._live_mlps


def test_static_charge_outputs_are_checked_before_the_call(pic):
    """pic_charges_get_static writes N0 doubles through each output it is given: a short,
    read-only, non-contiguous or non-float64 array is refused in the binding, before the
    library is called (a handle with a NULL simulation pointer would fail there)."""
    nodes, tris, be, bt = W.two_triangle_mesh()
    mesh = pic.pic_mesh_create(nodes, tris, be, bt)
    n0 = pic.pic_mesh_info(mesh)["n_nodes"]
    sim = pic.Sim.__new__(pic.Sim)
    sim.ptr, sim.mesh = None, mesh
    ro = np.zeros(n0)
    ro.flags.writeable = False
    bad = [np.zeros(n0 - 1), np.zeros(n0 + 1), np.zeros(n0, np.float32), ro,
           np.zeros(2 * n0)[::2], list(np.zeros(n0))]
    for x in bad:
        for pos in range(3):
            args = [None, None, None]
            args[pos] = x
            with pytest.raises(ValueError):
                pic.pic_charges_get_static(sim, *args)
