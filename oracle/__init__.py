"""FP64 CPU oracle for the stochastic Galerkin (SG) diffusion system of arXiv 1910.11505.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package: only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py`` use it.  It shares no code, table or constant generator with the CUDA library in
``paper_1910_11505_gb300/``; the two meet only on the seeded inputs of
``paper_1910_11505_gb300/workloads.py``, which hold none of the method's arithmetic.

Every function is a plain, slow, FP64 restatement of the paper's definitions (section and
equation cited in each docstring).  Library primitives (scipy sparse products, a triangular
solve, a bracketing root finder) are used as single steps; nothing is blocked, fused or
reordered beyond what the definitions state.

Parity status of each part (what pins it is listed in ``tests/test_oracle_pins.py``):
    KL modes, multi-indices, triple products, chaos coefficients, Q1 assembly, SG matvec,
    ILU(0), mean-based and field-split preconditioners, GMRES: pinned.
"""

from .sg_oracle import *  # noqa: F401,F403
