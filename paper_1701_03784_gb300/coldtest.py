"""Cold test of one slow-wave-structure period (the staircasing study of Sec. 5.3): the
cell between two ripple maxima with conducting end planes has, among its TM01-like
resonances, the 0 point (the pattern uniform in z) and the pi point (one half-wave along
z) of the periodic structure's dispersion.  The field solver rings the cell down from the
line integrals of a cylinder's TM010 + TM011 patterns and the two mode projections'
frequencies are fitted (two sinusoids plus offset by least squares, started from the
windowed spectrum's two largest peaks).  Conformal and staircased meshes of the same
spacing give the staircasing error."""
import numpy as np

from . import pic
from workloads.bwo import EPS0, MU0, C0
from workloads.fields import tm0np_edge_dofs
from workloads.meshes import sws_cell_mesh


def _frequency(t, a):
    """Frequency (Hz) of the strongest tone of a(t): two sinusoids and an offset fitted by
    least squares, started from the two largest peaks of the windowed spectrum (the other
    mode leaks into every projection)."""
    from scipy.optimize import least_squares
    n = len(a)
    spec = np.abs(np.fft.rfft((a - a.mean()) * np.hanning(n), 16 * n))
    freqs = np.fft.rfftfreq(16 * n, t[1] - t[0])
    k1 = 1 + int(np.argmax(spec[1:]))
    # the second peak: the largest at least two resolution widths away from the first
    far = np.abs(np.arange(len(spec)) - k1) > 2 * 16
    far[0] = False
    k2 = int(np.argmax(np.where(far, spec, 0.0)))
    w1, w2 = 2.0 * np.pi * freqs[k1], 2.0 * np.pi * freqs[k2]

    def res(p):
        return (p[0] * np.cos(p[2] * t) + p[1] * np.sin(p[2] * t) + p[3] * np.cos(p[5] * t)
                + p[4] * np.sin(p[5] * t) + p[6] - a)
    p = least_squares(res, [a.std(), 0.0, w1, 0.1 * a.std(), 0.0, w2, a.mean()],
                      x_scale="jac").x
    main = p[2] if np.hypot(p[0], p[1]) >= np.hypot(p[3], p[4]) else p[5]
    return main / (2.0 * np.pi)


def ring_down(n_tri, staircase, duration=1.5e-9, precision=pic.PIC_FP64, r0=15.0e-3,
              ripple=2.1e-3, period=7.5e-3, seed=1020):
    """(0-point, pi-point) frequencies in Hz of the cell meshed with about n_tri
    triangles, and the mesh size."""
    nodes, tris, be, bt = sws_cell_mesh(n_tri, seed, staircase, r0, ripple, period)
    mesh = pic.pic_mesh_create(nodes, tris, be, bt, eps0=EPS0, mu0=MU0, c=C0,
                               precision=precision)
    dt = 0.5 * pic.pic_spai_build(mesh, 2, 1e-4)
    edges = pic.pic_mesh_edges(mesh)
    P0 = tm0np_edge_dofs(nodes, edges, r0, period, 1, 0)
    P1 = tm0np_edge_dofs(nodes, edges, r0, period, 1, 1)
    sim = pic.pic_sim_create(mesh, dt, 0.0, 16)
    pic.pic_fields_set(sim, P0 + P1, np.zeros(len(tris)))
    n = int(duration / dt)
    a0, a1 = np.zeros(n), np.zeros(n)
    for k in range(n):
        E, _ = pic.pic_fields_get(sim)
        a0[k], a1[k] = E @ P0, E @ P1
        pic.pic_step(sim, 1)
    pic.pic_sim_destroy(sim)
    pic.pic_mesh_destroy(mesh)
    t = np.arange(n) * dt
    return _frequency(t, a0), _frequency(t, a1), len(tris)
