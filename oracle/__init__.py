"""FP64 CPU oracle of the online DMD hot path (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference arm of
``bench.py`` may import anything from this package.  The product path (the CUDA library
and its Python binding) never imports it and shares no code with it.

Modules
-------
odmd_ref   -- the incremental algorithm, step by step (Brand's rank-1 append, Sec. 2.3)
odmd_pairs -- the same update fed (x, y) pairs that need not be contiguous (the hybrid
              loop's reading in which only FOM steps update), with the hybrid loop
batch_dmd  -- exact DMD of the whole snapshot matrix (or of paired matrices), written
              from its definition (Sec. 2.3): the brute-force pin of the incremental
              paths on tiny inputs.

Parity status: every function here is pinned by tests in ``tests/test_oracle_*.py``
(brute force, closed forms, invariants).  Quantities that live in the noise subspace
(eigenvalues of modes with negligible amplitude) are parity unpinned by construction:
they are reported, not compared.
"""
from .odmd_ref import OnlineDMDRef
from .odmd_pairs import OnlineDMDPairsRef, hybrid_fom_updates
from .batch_dmd import BatchDMD, BatchPairDMD

__all__ = ["OnlineDMDRef", "OnlineDMDPairsRef", "hybrid_fom_updates", "BatchDMD", "BatchPairDMD"]
