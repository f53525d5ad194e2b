"""Plain FP64 CPU oracle of the FSLBM time step (arXiv 2207.13962).

Test infrastructure only: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may use it; the product path never does.
"""
from .oracle import (Oracle, build_oracle, collide, feq, k8_smooth, lattice, py_gradient,  # noqa: F401
                     reconstruct, seed_fill_front, select)
