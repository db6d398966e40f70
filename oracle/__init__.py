"""CPU FP64 oracle for the hydrothermal finite element step.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference leg of ``bench.py``; never by the product
path.  It shares no code with the CUDA library.

* ``fem``          -- assembled-matrix FE discretisation of Eq. 3 / Eq. 4
                      (head form), direct or tight-tolerance iterative solves.
* ``closed_forms`` -- analytic solutions used to pin ``fem``.
"""
from . import fem, closed_forms  # noqa: F401
