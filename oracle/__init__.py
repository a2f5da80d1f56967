"""FP64 CPU oracle of the SSGI hot path -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference leg may import this
package.  The library (paper_2504_01358_gb300/) never imports it, and it never imports the
library: the two share no code, only the data formats of include/ssgi.h and the seeded input
generators of ssgi_inputs/.

The arithmetic lives in ssgi_oracle.c (plain C, double precision); this module builds it with
gcc and wraps it with ctypes and numpy.
"""
from .oracle import *  # noqa: F401,F403
from .oracle import __all__  # noqa: F401
