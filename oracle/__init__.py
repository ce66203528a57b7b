"""FP64 CPU oracle of the boundary-element Poisson-Boltzmann hot path.

TEST INFRASTRUCTURE ONLY. The tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only users. The CUDA library and its
Python binding never import, link or execute anything here, and nothing here
imports them: the two share only the seeded input generators in ``synth``.

Parity pins: every function is checked in tests/ against something other than
itself (closed forms, invariants, brute force, library special cases); see
tests/test_oracle_*.py. Functions without such a pin say "parity unpinned".
"""
from .oracle import (CASES, FORMS, KCAL_PER_PAPER_UNIT, Operators, Physics, Plan, assemble,
                     assemble_rows, band_pair_count, gmres, interior_traces, pair_blocks, preconditioner,
                     reaction_potential, solve, source_projections, system)

__all__ = ["CASES", "FORMS", "KCAL_PER_PAPER_UNIT", "Operators", "Physics", "Plan", "assemble",
           "assemble_rows", "band_pair_count", "gmres", "interior_traces", "pair_blocks", "preconditioner",
           "reaction_potential", "solve", "source_projections", "system"]
