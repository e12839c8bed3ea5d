"""FP64 CPU oracle of the axisymmetric charge-conservative EM-PIC step (Na et al., 2017).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously-correct statement
of what the method computes; it exists to check the GPU library against.  Only the test
suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import it.
It shares no code with the GPU library (``paper_1701_03784_gb300``) and never imports it.

Layout:
  operators.py  mesh topology, incidence matrices (Sec. 3.1, App. D), Whitney/Hodge
                assembly (Eqs. dis_hodge_eps / dis_hodge_mu, App. B), SPAI (Sec. 3.1),
                stable time step, leapfrog field update (Eqs. full_d_dfl / full_d_dal),
                DCE / DGL residuals (Sec. 3.5, Sec. 5.1.1).
  particles.c   gather (Sec. 3.2), relativistic Boris push (Eqs. DNE / DLE), triangle
                walk, charge-conserving scatter (Eqs. charge / current), plain C, FP64.
  particles.py  ctypes wrapper around particles.c and the point-location used at
                injection.
  sim.py        one PIC cycle in the order of Sec. 3 (field, gather, push, scatter).
  sources.py    static gun field (Laplace problem), cathode emission with counter-based
                draws, planar space-charge-limited current (Secs. 5.2, 5.3).
  mlp.py        the surrogate network: forward, backward and Adam, written out plainly.
  port.py       output-port power: the Poynting flux of the discrete fields through a
                plane (Secs. 5.1, 5.1.1).

Every function's pin (what fixes it other than itself) is in tests/test_oracle_*.py;
tests/test_oracle_mutations.py plants one mistake at a time in a copy of a routine here
and checks that its pin fails.
"""
from .operators import Mesh, hodge_eps, hodge_mu_inv, spai, dt_stable, field_energy  # noqa: F401
from .sim import OracleSim  # noqa: F401
