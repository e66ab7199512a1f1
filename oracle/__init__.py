"""FP64 CPU oracle for the additive-kernel NFFT fast summation.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its ``cpu_baseline`` leg and its ``--impl reference`` arm) may
import anything from this package. The product package
``paper_2504_00480_gb300`` never imports it, and this package never imports
the product: the two share no code. Inputs come from the seeded generators in
``paper_2504_00480_gb300.inputs``, which hold none of the method's arithmetic.

See ``oracle.agp_oracle`` for the functions and the paper passage each one
follows, and the ``-m "not gpu"`` tests in ``tests/test_oracle_*.py`` for what
pins each function to something other than itself.
"""
from .agp_oracle import *  # noqa: F401,F403
