"""FP64 CPU oracle for the deep FBSDE solver (test infrastructure).

Plain NumPy, one statement per step of the method in arXiv 1910.11623.  Only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this package; the library never does, and this package imports nothing
from the library.
"""
from . import philox, fbsde  # noqa: F401
