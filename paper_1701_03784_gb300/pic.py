"""Thin ctypes binding of the C ABI in include/pic.h (same function names).

Argument marshalling only: every step of the method runs inside libpic_gb300.so.  The
library must have been built (``paper_1701_03784_gb300._build.build()``); importing this
module without it raises ImportError -- there is no fallback implementation.
"""
import atexit
import ctypes
import os
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpic_gb300.so")

PIC_OK, PIC_ERR_ARG, PIC_ERR_MESH, PIC_ERR_CUDA, PIC_ERR_UNSTABLE, PIC_ERR_TIMEOUT, \
    PIC_ERR_OOM, PIC_ERR_STATE = range(8)
PIC_BC_PEC, PIC_BC_AXIS, PIC_BC_ABSORB = 1, 2, 3
PIC_FP64, PIC_FP32 = 0, 1
PIC_PUSHER_BORIS, PIC_PUSHER_VAY = 0, 1
_STATUS = {0: "PIC_OK", 1: "PIC_ERR_ARG", 2: "PIC_ERR_MESH", 3: "PIC_ERR_CUDA",
           4: "PIC_ERR_UNSTABLE", 5: "PIC_ERR_TIMEOUT", 6: "PIC_ERR_OOM", 7: "PIC_ERR_STATE"}


class PicError(RuntimeError):
    def __init__(self, status, where, msg):
        super().__init__("%s: %s (%s)" % (where, msg, _STATUS.get(status, status)))
        self.status = status


class pic_units(ctypes.Structure):
    _fields_ = [("eps0", ctypes.c_double), ("mu0", ctypes.c_double), ("c", ctypes.c_double),
                ("precision", ctypes.c_int32), ("walk_cap", ctypes.c_int32)]


class pic_diag(ctypes.Structure):
    _fields_ = [("n_particles", ctypes.c_int64), ("n_absorbed", ctypes.c_int64),
                ("walk_overflows", ctypes.c_int64), ("n_crossings", ctypes.c_int64),
                ("n_steps", ctypes.c_int64), ("dce_max", ctypes.c_double),
                ("dce_nonzero", ctypes.c_int64), ("nr_dce_max", ctypes.c_double),
                ("dgl_drift", ctypes.c_double), ("field_energy", ctypes.c_double),
                ("kinetic_energy", ctypes.c_double), ("q_absorbed", ctypes.c_double),
                ("n_emitted", ctypes.c_int64), ("emit_dropped", ctypes.c_int64),
                ("steps_since_sort", ctypes.c_int64), ("sort_interval", ctypes.c_int64)]


class pic_emitter(ctypes.Structure):
    _fields_ = [("z", ctypes.c_double), ("rho0", ctypes.c_double), ("rho1", ctypes.c_double),
                ("per_step", ctypes.c_int64), ("u_normal", ctypes.c_double),
                ("u_thermal", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("q", ctypes.c_double), ("m", ctypes.c_double), ("w", ctypes.c_double)]


if not os.path.exists(LIB_PATH):
    raise ImportError("libpic_gb300.so is not built; run paper_1701_03784_gb300._build.build()")
_lib = ctypes.CDLL(LIB_PATH)

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_D = ctypes.c_double
_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_SIGS = {
    "pic_set_allocator": [_ALLOC_FN, _FREE_FN, _P],
    "pic_mesh_create": [_P, _I64, _P, _I64, _P, _P, _I64, ctypes.POINTER(pic_units), _P],
    "pic_mesh_info": [_P, _P, _P, _P, _P, _P],
    "pic_mesh_edges": [_P, _P],
    "pic_spai_build": [_P, _I32, _D, _P],
    "pic_spai_get": [_P, _P, _P, _P, _P],
    "pic_spai_info": [_P, _P, _P, _P],
    "pic_sim_create": [_P, _D, _D, _I64, _P],
    "pic_sim_set_sort_interval": [_P, _I32],
    "pic_sim_set_pusher": [_P, _I32],
    "pic_sim_set_wait_limit": [_P, _I64],
    "pic_static_potential": [_P, _I64, _P, _P, _P, _P, _P],
    "pic_sim_set_static_field": [_P, _P, _P],
    "pic_sim_set_emitter": [_P, ctypes.POINTER(pic_emitter), _P],
    "pic_sim_set_loss": [_P, _P, _P, _P],
    "pic_sim_set_probes": [_P, _I64, _P, _P, _P, _I32, _P, _I64, _I32, _P],
    "pic_probes_read": [_P, _P, _I64, _P, _P, _P],
    "pic_sim_set_ports": [_P, _I32, _P, _P, _P, _I64, _I32, _P],
    "pic_ports_read": [_P, _P, _I64, _P, _P, _P],
    "pic_sim_set_graph": [_P, _I32],
    "pic_sim_autotune": [_P, _I32, _P, _P],
    "pic_mlp_create": [_I32, _I32, _P, _I32, _P],
    "pic_mlp_param_count": [_P, _P],
    "pic_mlp_params_set": [_P, _P],
    "pic_mlp_params_get": [_P, _P],
    "pic_mlp_train": [_P, _P, _P, _I64, _I32, _I64, _D, ctypes.c_uint64, _P, _P],
    "pic_mlp_grad": [_P, _P, _P, _I64, _P, _P, _P],
    "pic_mlp_forward": [_P, _P, _P, _I64, _I32, _P],
    "pic_mlp_set_training": [_P, _I32],
    "pic_mlp_set_wait_limit": [_P, _I64],
    "pic_fields_set": [_P, _P, _P, _P],
    "pic_particles_inject": [_P, _I64, _P, _P, _P, _P, _P, _D, _D, _D, _P],
    "pic_step": [_P, _I64, _P],
    "pic_diagnostics": [_P, ctypes.POINTER(pic_diag), _P, _P, _P, _P],
    "pic_charges_get": [_P, _P, _P, _P, _P],
    "pic_charges_get_static": [_P, _P, _P, _P, _P],
    "pic_particles_count": [_P, _P, _P],
    "pic_particles_get": [_P, _I64, _P, _P, _P, _P, _P],
    "pic_particles_raw_bytes": [_P, _P],
    "pic_particles_raw_size": [_P, _I64, _P],
    "pic_particles_raw_get": [_P, _P, _I64, _P],
    "pic_particles_raw_set": [_P, _P, _I64, _P],
    "pic_step_host": [_P, _P, _I64, _I64, _P],
    "pic_kernel_timing": [_P, _I32, _P, _P, _P],
    "pic_launch_count": [_P],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int
_lib.pic_last_error.restype = ctypes.c_char_p
_lib.pic_last_error.argtypes = []
_lib.pic_sim_destroy.argtypes = [_P]
_lib.pic_sim_destroy.restype = None
_lib.pic_mesh_destroy.argtypes = [_P]
_lib.pic_mesh_destroy.restype = None
_lib.pic_mlp_destroy.argtypes = [_P]
_lib.pic_mlp_destroy.restype = None

EXPORTED = sorted(list(_SIGS) + ["pic_last_error", "pic_sim_destroy", "pic_mesh_destroy",
                                  "pic_mlp_destroy"])


def _check(status, where):
    if status != PIC_OK:
        raise PicError(status, where, pic_last_error())


def _arr(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _stream(stream):
    """CUDA stream handle: an int, a torch.cuda.Stream, or None for torch's current stream
    (the legacy default stream when torch is absent)."""
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def pic_last_error():
    return _lib.pic_last_error().decode()


# ---- device memory from PyTorch's caching allocator ------------------------------------
_torch_hooks = None


def use_torch_allocator():
    """Route the library's device allocations through torch.cuda's caching allocator."""
    global _torch_hooks
    import torch

    def _alloc(nbytes, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes))
        except RuntimeError:
            return None

    def _free(ptr, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    hooks = (_ALLOC_FN(_alloc), _FREE_FN(_free))
    _check(_lib.pic_set_allocator(hooks[0], hooks[1], None), "pic_set_allocator")
    _torch_hooks = hooks


def pic_set_allocator(alloc=None, free=None):
    """Install ctypes-compatible alloc/free callbacks, or restore cudaMalloc (no args)."""
    global _torch_hooks
    if alloc is None:
        _check(_lib.pic_set_allocator(_ALLOC_FN(), _FREE_FN(), None), "pic_set_allocator")
        _torch_hooks = None
        return
    hooks = (_ALLOC_FN(alloc), _FREE_FN(free))
    _check(_lib.pic_set_allocator(hooks[0], hooks[1], None), "pic_set_allocator")
    _torch_hooks = hooks


# ---- handles -------------------------------------------------------------------------
class Mesh:
    def __init__(self, ptr, precision):
        self.ptr = ptr
        self.precision = precision

    def __del__(self):
        if getattr(self, "ptr", None):
            _lib.pic_mesh_destroy(self.ptr)
            self.ptr = None


class Sim:
    def __init__(self, ptr, mesh):
        self.ptr = ptr
        self.mesh = mesh          # the mesh must outlive the simulation
        # the library keeps the allocator hooks a simulation was created with and calls
        # them when it frees its memory: keep their trampolines alive as long
        self._hooks = _torch_hooks
        _live_sims.add(self)

    def __del__(self):
        if getattr(self, "ptr", None):
            _lib.pic_sim_destroy(self.ptr)
            self.ptr = None


_live_sims = weakref.WeakSet()
_live_mlps = weakref.WeakSet()


@atexit.register
def _destroy_live_sims():
    # free device memory while the allocator callbacks (torch) are still alive
    for s in list(_live_sims):
        if s.ptr:
            _lib.pic_sim_destroy(s.ptr)
            s.ptr = None
    for n in list(_live_mlps):
        if n.ptr:
            _lib.pic_mlp_destroy(n.ptr)
            n.ptr = None


def pic_mesh_create(nodes_zr, tris, bedge_nodes, bedge_tag, eps0=1.0, mu0=1.0, c=None,
                    precision=PIC_FP32, walk_cap=0):
    nodes_zr = _arr(nodes_zr, np.float64)
    tris = _arr(tris, np.int32)
    bedge_nodes = _arr(bedge_nodes, np.int32)
    bedge_tag = _arr(bedge_tag, np.int32)
    if c is None:
        c = 1.0 / np.sqrt(eps0 * mu0)
    u = pic_units(eps0, mu0, c, precision, walk_cap)
    out = ctypes.c_void_p()
    _check(_lib.pic_mesh_create(_ptr(nodes_zr), len(nodes_zr), _ptr(tris), len(tris),
                                _ptr(bedge_nodes), _ptr(bedge_tag), len(bedge_tag),
                                ctypes.byref(u), ctypes.byref(out)), "pic_mesh_create")
    return Mesh(out, precision)


def pic_mesh_info(mesh):
    v = [ctypes.c_int64() for _ in range(5)]
    _check(_lib.pic_mesh_info(mesh.ptr, *[ctypes.byref(x) for x in v]), "pic_mesh_info")
    return dict(zip(["n_nodes", "n_edges", "n_tris", "n_free_edges", "spai_nnz"],
                    [x.value for x in v]))


def pic_mesh_edges(mesh):
    n = pic_mesh_info(mesh)["n_edges"]
    out = np.zeros((n, 2), np.int32)
    _check(_lib.pic_mesh_edges(mesh.ptr, _ptr(out)), "pic_mesh_edges")
    return out


def pic_spai_build(mesh, pattern_level=2, drop_tol=1e-4):
    dt = ctypes.c_double()
    _check(_lib.pic_spai_build(mesh.ptr, pattern_level, drop_tol, ctypes.byref(dt)),
           "pic_spai_build")
    return dt.value


def pic_spai_info(mesh):
    """{nnz, residual_rms, residual_max} of M against star_eps on the free edges."""
    nnz = _I64()
    rms, mx = ctypes.c_double(), ctypes.c_double()
    _check(_lib.pic_spai_info(mesh.ptr, ctypes.byref(nnz), ctypes.byref(rms), ctypes.byref(mx)),
           "pic_spai_info")
    return {"nnz": nnz.value, "residual_rms": rms.value, "residual_max": mx.value}


def pic_spai_get(mesh):
    info = pic_mesh_info(mesh)
    nf, nnz = info["n_free_edges"], info["spai_nnz"]
    fe = np.zeros(nf, np.int32)
    ip = np.zeros(nf + 1, np.int64)
    ix = np.zeros(nnz, np.int32)
    vv = np.zeros(nnz, np.float64)
    _check(_lib.pic_spai_get(mesh.ptr, _ptr(fe), _ptr(ip), _ptr(ix), _ptr(vv)), "pic_spai_get")
    return fe, ip, ix, vv


def pic_sim_create(mesh, dt, bz_guide=0.0, max_particles=0, torch_memory=True):
    if torch_memory and _torch_hooks is None:
        try:
            import torch
            if torch.cuda.is_available():
                use_torch_allocator()
        except ImportError:
            pass
    out = ctypes.c_void_p()
    _check(_lib.pic_sim_create(mesh.ptr, dt, bz_guide, int(max_particles), ctypes.byref(out)),
           "pic_sim_create")
    return Sim(out, mesh)


def pic_sim_set_sort_interval(sim, interval):
    _check(_lib.pic_sim_set_sort_interval(sim.ptr, interval), "pic_sim_set_sort_interval")


def pic_static_potential(mesh, held_nodes, held_phi, charge=None):
    """(phi on nodes, E_static on edges): phi held at held_nodes, discrete Poisson problem
    with the node charges (per radian; None: none) elsewhere (Sec. 5.3)."""
    held_nodes = _arr(held_nodes, np.int32)
    held_phi = _arr(np.broadcast_to(held_phi, held_nodes.shape), np.float64)
    Q = None if charge is None else _arr(charge, np.float64)
    info = pic_mesh_info(mesh)
    phi = np.zeros(info["n_nodes"])
    E = np.zeros(info["n_edges"])
    _check(_lib.pic_static_potential(mesh.ptr, len(held_nodes), _ptr(held_nodes),
                                     _ptr(held_phi), _ptr(Q), _ptr(phi), _ptr(E)),
           "pic_static_potential")
    return phi, E


def pic_sim_set_static_field(sim, E_static, stream=None):
    """Static field added at the gather (None removes it)."""
    Es = None if E_static is None else _arr(E_static, np.float64)
    _check(_lib.pic_sim_set_static_field(sim.ptr, _ptr(Es), _stream(stream)),
           "pic_sim_set_static_field")


def pic_sim_set_emitter(sim, z, rho0, rho1, per_step, u_normal, u_thermal, seed, q, m, w,
                        stream=None):
    """Emit per_step particles at the start of every step (see pic.h); per_step=None
    stops emission."""
    if per_step is None:
        _check(_lib.pic_sim_set_emitter(sim.ptr, None, _stream(stream)), "pic_sim_set_emitter")
        return
    e = pic_emitter(z, rho0, rho1, per_step, u_normal, u_thermal, seed, q, m, w)
    _check(_lib.pic_sim_set_emitter(sim.ptr, ctypes.byref(e), _stream(stream)),
           "pic_sim_set_emitter")


def pic_sim_set_loss(sim, sigma_e, sigma_m, stream=None):
    """Absorbing layer: conductivity per edge (S/m) and magnetic conductivity per face
    (ohm/m); both None makes the fields lossless again."""
    se = None if sigma_e is None else _arr(sigma_e, np.float64)
    sm = None if sigma_m is None else _arr(sigma_m, np.float64)
    _check(_lib.pic_sim_set_loss(sim.ptr, _ptr(se), _ptr(sm), _stream(stream)),
           "pic_sim_set_loss")


def pic_sim_set_probes(sim, face, group, weight, power, capacity, every, stream=None):
    """Device-recorded field sums (see pic.h); face/group/weight per entry, power per
    group (1: sum w B, 2: sum w B^2).  Empty face removes the probes."""
    face = _arr(face, np.int32)
    group = _arr(group, np.int32)
    weight = _arr(weight, np.float64)
    power = _arr(power, np.int32)
    _check(_lib.pic_sim_set_probes(sim.ptr, len(face), _ptr(face), _ptr(group), _ptr(weight),
                                   len(power), _ptr(power), int(capacity), int(every),
                                   _stream(stream)), "pic_sim_set_probes")
    sim.probe_groups = len(power)
    sim.probe_capacity = int(capacity)


def pic_probes_read(sim, stream=None):
    """(records x groups array of the sums recorded since the last read, dropped count)."""
    out = np.zeros((getattr(sim, "probe_capacity", 0), getattr(sim, "probe_groups", 0)))
    n, d = _I64(), _I64()
    _check(_lib.pic_probes_read(sim.ptr, _ptr(out), len(out), ctypes.byref(n),
                                ctypes.byref(d), _stream(stream)), "pic_probes_read")
    return out[:n.value].copy(), d.value


def pic_sim_set_ports(sim, z, rho0, rho1, capacity, every=1, stream=None):
    """Output-port power (Poynting flux through planes z[k], rho0[k]..rho1[k]) recorded on
    the device every `every` steps; z = None removes the ports."""
    if z is None:
        _check(_lib.pic_sim_set_ports(sim.ptr, 0, None, None, None, 1, 1, _stream(stream)),
               "pic_sim_set_ports")
        sim._ports = 0
        return
    z = _arr(np.atleast_1d(z), np.float64)
    r0 = _arr(np.broadcast_to(rho0, z.shape), np.float64)
    r1 = _arr(np.broadcast_to(rho1, z.shape), np.float64)
    _check(_lib.pic_sim_set_ports(sim.ptr, len(z), _ptr(z), _ptr(r0), _ptr(r1), int(capacity),
                                  int(every), _stream(stream)), "pic_sim_set_ports")
    sim._ports = len(z)
    sim._port_cap = int(capacity)


def pic_ports_read(sim, stream=None):
    """(records x n_ports array of port powers since the last read, records dropped)."""
    n = getattr(sim, "_ports", 0)
    cap = getattr(sim, "_port_cap", 0)
    out = np.zeros((max(cap, 1), max(n, 1)))
    nr, nd = ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.pic_ports_read(sim.ptr, _ptr(out), cap, ctypes.byref(nr), ctypes.byref(nd),
                               _stream(stream)), "pic_ports_read")
    return out[:nr.value, :n].copy(), nd.value


def pic_sim_set_pusher(sim, pusher):
    """PIC_PUSHER_BORIS (default) or PIC_PUSHER_VAY: the velocity update of Eq. DLE."""
    _check(_lib.pic_sim_set_pusher(sim.ptr, pusher), "pic_sim_set_pusher")


def pic_sim_set_wait_limit(sim, polls):
    """Polls before a tile-pipeline wait of the particle kernel gives up (default 16384)."""
    _check(_lib.pic_sim_set_wait_limit(sim.ptr, int(polls)), "pic_sim_set_wait_limit")


def pic_sim_set_graph(sim, enable=True):
    _check(_lib.pic_sim_set_graph(sim.ptr, 1 if enable else 0), "pic_sim_set_graph")


class pic_tuning(ctypes.Structure):
    _fields_ = [("sort_interval", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("field_block", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("ms_per_step", ctypes.c_double)]


def pic_sim_autotune(sim, trial_steps=32, stream=None):
    """Pick the launch shapes (re-sort interval, particle-kernel CTAs per SM, field-kernel
    block size) by timing trial steps; the simulation advances by up to 14 x trial_steps."""
    t = pic_tuning()
    _check(_lib.pic_sim_autotune(sim.ptr, int(trial_steps), ctypes.byref(t), _stream(stream)),
           "pic_sim_autotune")
    return {k: getattr(t, k) for k, _ in pic_tuning._fields_ if k != "pad"}


def pic_fields_set(sim, E=None, B=None, stream=None):
    E = None if E is None else _arr(E, np.float64)
    B = None if B is None else _arr(B, np.float64)
    _check(_lib.pic_fields_set(sim.ptr, _ptr(E), _ptr(B), _stream(stream)), "pic_fields_set")


def pic_particles_inject(sim, z, rho, u_rho, u_phi, u_z, q, m, weight, stream=None):
    z, rho, u_rho, u_phi, u_z = (_arr(x, np.float64) for x in (z, rho, u_rho, u_phi, u_z))
    n = len(z)
    assert all(len(x) == n for x in (rho, u_rho, u_phi, u_z))
    _check(_lib.pic_particles_inject(sim.ptr, n, _ptr(z), _ptr(rho), _ptr(u_rho), _ptr(u_phi),
                                     _ptr(u_z), q, m, weight, _stream(stream)),
           "pic_particles_inject")


def pic_step(sim, n_steps=1, stream=None):
    _check(_lib.pic_step(sim.ptr, int(n_steps), _stream(stream)), "pic_step")


def pic_diagnostics(sim, fields=False, stream=None):
    d = pic_diag()
    info = pic_mesh_info(sim.mesh)
    E = B = J = None
    if fields:
        E = np.zeros(info["n_edges"])
        B = np.zeros(info["n_tris"])
        J = np.zeros(info["n_edges"])
    _check(_lib.pic_diagnostics(sim.ptr, ctypes.byref(d), _ptr(E), _ptr(B), _ptr(J),
                                _stream(stream)), "pic_diagnostics")
    out = {k: getattr(d, k) for k, _ in pic_diag._fields_}
    if fields:
        out.update(E=E, B=B, J=J)
    return out


def pic_fields_get(sim, stream=None):
    """(E on edges, B on faces) as float64 arrays: pic_diagnostics without its reductions."""
    info = pic_mesh_info(sim.mesh)
    E = np.zeros(info["n_edges"])
    B = np.zeros(info["n_tris"])
    _check(_lib.pic_diagnostics(sim.ptr, None, _ptr(E), _ptr(B), None, _stream(stream)),
           "pic_diagnostics")
    return E, B


def pic_charges_get_static(sim, Q=None, Q_prev=None, Q_absorbed=None, stream=None):
    """pic_charges_get for callers that must not allocate device memory (the library's
    fixed scratch is used instead; meshes up to 131072 nodes).  The output arrays are the
    caller's (float64, N0 each) and are filled in place; None skips one."""
    n0 = pic_mesh_info(sim.mesh)["n_nodes"]
    for name, x in (("Q", Q), ("Q_prev", Q_prev), ("Q_absorbed", Q_absorbed)):
        # the library writes N0 doubles through each non-NULL pointer: anything that is not
        # a writeable, C-contiguous float64 array of exactly N0 elements is refused here,
        # before the call
        if x is None:
            continue
        if not isinstance(x, np.ndarray):
            raise ValueError("pic_charges_get_static: %s must be a numpy array" % name)
        if x.dtype != np.float64 or not x.flags.c_contiguous or not x.flags.writeable:
            raise ValueError("pic_charges_get_static: %s must be a writeable, C-contiguous "
                             "float64 array" % name)
        if x.size != n0:
            raise ValueError("pic_charges_get_static: %s has %d elements, the mesh has %d "
                             "nodes" % (name, x.size, n0))
    _check(_lib.pic_charges_get_static(sim.ptr, _ptr(Q), _ptr(Q_prev), _ptr(Q_absorbed),
                                       _stream(stream)), "pic_charges_get_static")
    return Q, Q_prev, Q_absorbed


def pic_charges_get(sim, stream=None):
    n0 = pic_mesh_info(sim.mesh)["n_nodes"]
    Q, Qp, Qa = np.zeros(n0), np.zeros(n0), np.zeros(n0)
    _check(_lib.pic_charges_get(sim.ptr, _ptr(Q), _ptr(Qp), _ptr(Qa), _stream(stream)),
           "pic_charges_get")
    return Q, Qp, Qa


def pic_particles_count(sim, stream=None):
    n = ctypes.c_int64()
    _check(_lib.pic_particles_count(sim.ptr, ctypes.byref(n), _stream(stream)),
           "pic_particles_count")
    return n.value


def pic_particles_get(sim, stream=None):
    n = pic_particles_count(sim, stream)
    pid = np.zeros(n, np.int64)
    tri = np.zeros(n, np.int32)
    lam = np.zeros((n, 3))
    u = np.zeros((n, 3))
    _check(_lib.pic_particles_get(sim.ptr, n, _ptr(pid), _ptr(tri), _ptr(lam), _ptr(u),
                                  _stream(stream)), "pic_particles_get")
    return dict(pid=pid, tri=tri, lam=lam, u=u)


def pic_particles_raw_bytes(sim):
    b = ctypes.c_int64()
    _check(_lib.pic_particles_raw_bytes(sim.ptr, ctypes.byref(b)), "pic_particles_raw_bytes")
    return b.value


def pic_particles_raw_size(sim, n_slots):
    """Bytes of a raw host buffer of n_slots slots (each array starts on a 128-byte
    boundary: the per-array stride is n_slots rounded up to 32)."""
    b = ctypes.c_int64()
    _check(_lib.pic_particles_raw_size(sim.ptr, int(n_slots), ctypes.byref(b)),
           "pic_particles_raw_size")
    return b.value


def pic_particles_raw_get(sim, host_ptr, n_slots, stream=None):
    """host_ptr: address (int) of a page-locked buffer of pic_particles_raw_size bytes."""
    _check(_lib.pic_particles_raw_get(sim.ptr, ctypes.c_void_p(host_ptr), int(n_slots),
                                      _stream(stream)), "pic_particles_raw_get")


def pic_particles_raw_set(sim, host_ptr, n_slots, stream=None):
    _check(_lib.pic_particles_raw_set(sim.ptr, ctypes.c_void_p(host_ptr), int(n_slots),
                                      _stream(stream)), "pic_particles_raw_set")


def pic_step_host(sim, host_ptr, n_slots, n_steps=1, stream=None):
    """n_steps steps with the raw state in the page-locked host buffer at host_ptr
    (pic_particles_raw_size bytes): uploaded, stepped and written back every step."""
    _check(_lib.pic_step_host(sim.ptr, ctypes.c_void_p(host_ptr), int(n_slots), int(n_steps),
                              _stream(stream)), "pic_step_host")


def pic_kernel_timing(sim, enable=True, stream=None):
    """Returns (milliseconds, launches) of the particle kernel since the last call and
    turns the per-launch CUDA-event timing on or off."""
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(_lib.pic_kernel_timing(sim.ptr, 1 if enable else 0, ctypes.byref(ms), ctypes.byref(n),
                                  _stream(stream)), "pic_kernel_timing")
    return ms.value, n.value


def pic_launch_count():
    """Kernels the library has enqueued for execution in this process (graph replays
    count their kernels)."""
    n = ctypes.c_int64()
    _check(_lib.pic_launch_count(ctypes.byref(n)), "pic_launch_count")
    return n.value


def pic_sim_destroy(sim):
    if sim.ptr:
        _lib.pic_sim_destroy(sim.ptr)
        sim.ptr = None


def pic_mesh_destroy(mesh):
    if mesh.ptr:
        _lib.pic_mesh_destroy(mesh.ptr)
        mesh.ptr = None


# ---- surrogate network ensemble ------------------------------------------------------------

class Mlp:
    def __init__(self, ptr, members, sizes):
        self.ptr = ptr
        self.members = members
        self.sizes = tuple(sizes)
        self._hooks = _torch_hooks   # allocator trampolines the library keeps (see Sim)
        _live_mlps.add(self)

    def __del__(self):
        if getattr(self, "ptr", None):
            _lib.pic_mlp_destroy(self.ptr)
            self.ptr = None


def _dev(t, what):
    """Address of a contiguous FP32 CUDA tensor."""
    import torch
    assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous(), what
    return ctypes.c_void_p(t.data_ptr())


def pic_mlp_create(n_members, sizes, max_batch):
    sz = np.ascontiguousarray(sizes, dtype=np.int32)
    out = _P()
    _check(_lib.pic_mlp_create(int(n_members), len(sz) - 1, _ptr(sz), int(max_batch),
                               ctypes.byref(out)), "pic_mlp_create")
    return Mlp(out, int(n_members), sz)


def pic_mlp_param_count(m):
    n = ctypes.c_int64()
    _check(_lib.pic_mlp_param_count(m.ptr, ctypes.byref(n)), "pic_mlp_param_count")
    return n.value


def pic_mlp_params_set(m, params):
    p = np.ascontiguousarray(params, dtype=np.float64)
    assert p.size == m.members * pic_mlp_param_count(m)
    _check(_lib.pic_mlp_params_set(m.ptr, _ptr(p)), "pic_mlp_params_set")


def pic_mlp_params_get(m):
    p = np.zeros((m.members, pic_mlp_param_count(m)))
    _check(_lib.pic_mlp_params_get(m.ptr, _ptr(p)), "pic_mlp_params_get")
    return p


def pic_mlp_train(m, X, T, batch, steps, lr=1e-3, seed=0, stream=None):
    """Adam steps on minibatches of the device rows X (n x in) and T (n x out); returns each
    member's loss on its last minibatch."""
    loss = np.zeros(m.members)
    _check(_lib.pic_mlp_train(m.ptr, _dev(X, "X"), _dev(T, "T"), X.shape[0], int(batch),
                              int(steps), float(lr), int(seed), _ptr(loss), _stream(stream)),
           "pic_mlp_train")
    return loss


def pic_mlp_grad(m, X, T, stream=None):
    g = np.zeros((m.members, pic_mlp_param_count(m)))
    loss = np.zeros(m.members)
    _check(_lib.pic_mlp_grad(m.ptr, _dev(X, "X"), _dev(T, "T"), X.shape[0], _ptr(g), _ptr(loss),
                             _stream(stream)), "pic_mlp_grad")
    return g, loss


def pic_mlp_set_wait_limit(m, polls):
    """Polls before a wait of the tensor-core inference kernel gives up (default 4194304)."""
    _check(_lib.pic_mlp_set_wait_limit(m.ptr, int(polls)), "pic_mlp_set_wait_limit")


def pic_mlp_set_training(m, tensor_cores):
    """Training and gradient products on the tensor cores (BF16 operands) or not."""
    _check(_lib.pic_mlp_set_training(m.ptr, 1 if tensor_cores else 0), "pic_mlp_set_training")


def pic_mlp_forward(m, X, tensor_cores=False, out=None, stream=None):
    """Device outputs (members x n x out, FP32) for the device rows X (n x in)."""
    import torch
    n = X.shape[0]
    Y = out if out is not None else torch.empty((m.members, n, int(m.sizes[-1])),
                                                 dtype=torch.float32, device=X.device)
    _check(_lib.pic_mlp_forward(m.ptr, _dev(X, "X"), _dev(Y, "Y"), n, 1 if tensor_cores else 0,
                                _stream(stream)), "pic_mlp_forward")
    return Y
