"""Plain FP64 CPU oracle for Wannier interpolation of e-ph matrix elements.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it.  The product (the CUDA library
and its Python binding) never imports, links or calls anything here, and this
package imports nothing from the product.
"""
from .eph_oracle import *  # noqa: F401,F403
