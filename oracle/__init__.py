"""fg21 oracle -- TEST INFRASTRUCTURE ONLY.

A plain, slow FP64 CPU statement of the region-partitioned global-21cm
likelihood (arXiv 2603.13196, Secs. 2.1-2.3 and 4), independent of the CUDA
library: the two share no code, and neither imports the other.  Only the test
suite, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` may
import or execute anything in this package; the product path never does.

Parity status: every routine here is pinned by a `-m "not gpu"` test against
a closed form, an invariant, a library routine or brute force (see
tests/test_oracle_pins.py); none is "parity unpinned" except the synthetic
input geometry, which is a definition rather than a result.
"""
from .oracle import *  # noqa: F401,F403
