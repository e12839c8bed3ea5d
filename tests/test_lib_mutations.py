"""Planted mistakes in the library's host code: each case copies the package into a
temporary folder, changes one term of a host routine (the Hodge quadrature, the SPAI
symmetrisation, the static field's edge values), builds that copy, and checks that its
results leave the oracle's, by far more than the parity tolerance, while an unchanged
copy matches.  This shows that the host parity tests constrain the library, not only
the oracle.  CPU only (the calls touched here do no device work)."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = "paper_1701_03784_gb300"

_CHILD = r'''
import sys
sys.path[:0] = [sys.argv[1], sys.argv[2]]
import numpy as np
import paper_1701_03784_gb300 as pkg
assert pkg.__file__.startswith(sys.argv[1])
pkg.build()
from paper_1701_03784_gb300 import pic
import workloads as W
from oracle.operators import Mesh, hodge_eps, spai
from oracle import sources as S

nodes, tris, be, bt = W.cavity_mesh(n_tri=600, seed=3)
om = Mesh(nodes, tris, be, bt)
m = pic.pic_mesh_create(nodes, tris, be, bt)
pic.pic_spai_build(m, 2, 1e-4)
_, ip, ix, vv = pic.pic_spai_get(m)
M = spai(om, hodge_eps(om), 2, 1e-4).tocsr()
M.sort_indices()
same = np.array_equal(ip, M.indptr) and np.array_equal(ix, M.indices)
d_spai = np.abs(vv - M.data).max() / np.abs(M.data).max() if same else np.inf
held = np.flatnonzero((om.nodes[:, 0] == 0.0) | (om.nodes[:, 0] == 1.0))
phi_l, E_l = pic.pic_static_potential(m, held, 3.0 * om.nodes[held, 0])
_, E_o = S.static_potential(om, hodge_eps(om), held, 3.0 * om.nodes[held, 0])
d_static = np.abs(E_l - E_o).max() / np.abs(E_o).max()
print("spai %.3e static %.3e" % (d_spai, d_static))
'''

CASES = [
    ("unchanged", None, None, None),
    ("Hodge quadrature: a wrong centre weight", "mesh.cpp",
     "w[q++] = 9.0 / 40.0;", "w[q++] = 9.0 / 41.0;"),
    ("SPAI: the transposed half left out", "spai.cpp",
     "trip.push_back({(uint64_t)j * (uint64_t)nf + (uint64_t)rv.first, 0.5 * rv.second});",
     "trip.push_back({(uint64_t)j * (uint64_t)nf + (uint64_t)rv.first, 0.0 * rv.second});"),
    ("static field: head minus tail", "sources.cpp",
     "E_out[e] = phi[m.edge_nodes[2 * e]] - phi[m.edge_nodes[2 * e + 1]];",
     "E_out[e] = phi[m.edge_nodes[2 * e + 1]] - phi[m.edge_nodes[2 * e]];"),
]


def _copy_package(dst):
    src = os.path.join(ROOT, PKG)
    os.makedirs(os.path.join(dst, PKG, "csrc"))
    for f in os.listdir(src):
        if f.endswith(".py"):
            shutil.copy(os.path.join(src, f), os.path.join(dst, PKG, f))
    for f in os.listdir(os.path.join(src, "csrc")):
        shutil.copy(os.path.join(src, "csrc", f), os.path.join(dst, PKG, "csrc", f))
    shutil.copytree(os.path.join(ROOT, "include"), os.path.join(dst, "include"))


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_in_the_host_library_breaks_parity(case, tmp_path):
    if shutil.which(os.environ.get("NVCC", "nvcc")) is None:
        pytest.skip("nvcc not available")
    name, src, old, new = case
    _copy_package(str(tmp_path))
    if src is not None:
        path = tmp_path / PKG / "csrc" / src
        text = path.read_text()
        assert text.count(old) == 1, old
        path.write_text(text.replace(old, new))
    script = tmp_path / "child.py"
    script.write_text(_CHILD)
    out = subprocess.run([sys.executable, str(script), str(tmp_path), ROOT],
                         capture_output=True, text=True, timeout=600, cwd=str(tmp_path))
    assert out.returncode == 0, out.stderr[-3000:]
    words = out.stdout.split()
    d_spai, d_static = float(words[1]), float(words[3])
    if src is None:
        assert d_spai < 1e-9 and d_static < 1e-9
    elif src == "sources.cpp":
        assert d_static > 1e-3
    else:
        assert d_spai > 1e-3
