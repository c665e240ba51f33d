"""FP64 CPU oracle for batched GP-GOMEA fitness evaluation.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run anything in this package.
The library (``paper_2605_30954_gb300``) never imports it, and it shares no
code, header, table or constant with the library: the template opcodes below
are written out by hand from the library's documented interface.

What it computes (plain definitions, slow on purpose):

* the value of a template tree's active expression at every dataset row,
  evaluated recursively in FP64 from the root; intron nodes are never
  visited (Section 3.1 and Fig. 1 of the paper);
* the post-order (RPN) sequence of the active nodes (Section 3.2,
  "Data Structure of Individuals") and the paper's (T, V) array encoding;
* MSE (Eq. 1), NMSE (Eq. 2) and the linearly scaled MSE
  ``min_{a,b} mean((y - a - b f)^2)`` with the least-squares a*, b*
  (Keijzer's linear scaling, which the paper names but does not define);
* the reverse-mode FP64 gradient of (scaled) MSE with respect to every ERC
  constant, and central finite differences of the same quantity;
* an FP32-emulating evaluator (every node rounded to float32, float32 libm)
  and a first-order condition bound, which the tests use only to flag rows
  and trials whose FP32 value is ill-conditioned;
* one GOM step of Algorithm 1 (donor copy, the "changed" test, accept or
  revert) in ``oracle.gom``.

Parity pins (tests/test_oracle_pins.py) tie every function here to the
paper's worked example, closed forms, library special cases and brute force.
"""
from .gp import *  # noqa: F401,F403
from . import gom  # noqa: F401
