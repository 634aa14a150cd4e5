"""CPU oracle for the block-forest AMR lattice Boltzmann method (arXiv 2308.08085).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 restatement of
what the paper's method computes, written from the paper's text.  It shares no
code with the CUDA library under ``paper_2308_08085_gb300`` and imports nothing
from it.  Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
/ ``--impl reference`` legs of ``bench.py`` may import it; the product path must
never route through it.

Modules
-------
lattice   velocity sets, weights, equilibrium, moments (Section 2)
uniform   dense uniform-grid LBM used to pin the forest solver (Section 2)
forest    block forest: root grid, connectivity by geometry, cell classes,
          refinement/coarsening with ID sets and the gap set (Section 3.2-3.3)
solver    forest LBM: collide/stream with boundary conditions, coarse-to-fine
          interpolation, fine-to-coarse averaging, recursive level step,
          pre-adapt synchronisation, vorticity criterion, force probe, MLUPS
          (Sections 3.4, 4, 5.1, 5.3)

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
invariants or brute force; functions without such a pin say "parity unpinned"
in their docstring.
"""
