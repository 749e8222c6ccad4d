"""FP64 CPU oracle for GOFMM (geometry-oblivious FMM, Yu, Levitt, Reiz, Biros,
SC'17).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import or run anything in this
package.  The native library never calls it, and it never calls the native
library: the two share no code.
"""
from .gofmm_oracle import *  # noqa: F401,F403
