"""Plain FP64 CPU oracle for many-particle CTQW propagation.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run anything in this package.
The product path (the CUDA library and its Python binding) never calls it,
and it shares no code with the product path: the one module both sides import
is ``ctqw_workloads`` (seeded uniform draws and workload shapes, no arithmetic
of the method).

Every function cites the passage of the paper it follows (Piccinini et al.,
"GPU-accelerated algorithms for many-particle continuous-time quantum walks",
arXiv:1612.00746).  Parity status: every function is pinned by a closed form,
a brute-force construction or an invariant in ``tests/test_oracle_pins.py``;
none is "parity unpinned".
"""
from .ctqw_oracle import *  # noqa: F401,F403
