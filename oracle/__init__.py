"""CPU oracle for Panorama exact kNN refinement -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference arm may import, call, link or execute anything in this package.  The
CUDA library never does, and nothing here imports the library: the two share
no code.  The only common module is ``synth`` (seeded input draws, none of the
method's arithmetic).

What is here, all in FP64 unless stated:

* ``reference.py`` -- the method's mathematics written out plainly: PCA fit
  (Section 4.1), the level decomposition and bounds (Eq. 1-4), Algorithm 1
  (batched iterative refinement), IVF assignment/probing (Section 6.1), the
  energy-compaction diagnostic E(m) and its decay alpha (Section 4.1), and the
  brute-force definition of the answer (Problem 1).
* ``pq.py`` -- IVFPQ Panorama: spectrum shaping (Section 4.3, Robin Hood
  inter-level shaping and intra-level Haar isotropisation), product
  quantisation of IVF residuals, asymmetric distances, the Eq. 3 bounds in
  partial-distance form and Algorithm 1 over asymmetric distances
  (Section 6.3).
* ``topk.c`` -- the brute-force answer of Problem 1 over an IVF candidate set,
  plain C, FP64, one thread per host core; compiled by ``build_native()``.

Parity status per function (what pins it) is listed in the module docstrings.
"""
from .reference import *  # noqa: F401,F403
from .native import build_native, ivf_topk  # noqa: F401
