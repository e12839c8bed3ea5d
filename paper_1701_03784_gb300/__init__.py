"""GB300 (sm_103a) library for the per-step particle loop of the axisymmetric
charge-conservative EM-PIC method on unstructured meshes (Na et al., 2017).

The compute path lives in the C-ABI shared library ``libpic_gb300.so`` (include/pic.h);
``paper_1701_03784_gb300.pic`` is its thin ctypes binding and raises ImportError when
the library has not been built (``paper_1701_03784_gb300.build()``).
"""
from ._build import build  # noqa: F401
