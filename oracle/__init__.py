"""Plain FP64 CPU oracle for MORE-Stress (arXiv 2411.12690).

TEST INFRASTRUCTURE ONLY. This package exists so that tests can check the CUDA
library against an independent, slow, obviously correct implementation of the
same mathematics. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs
of ``bench.py`` (``cpu_baseline`` and ``--impl reference``) may import it. The
product package ``paper_2411_12690_gb300`` never imports it and shares no code,
table or constant with it.

* ``oracle.fem`` -- O-FEM: the full fine-mesh Q1-hex thermoelastic model (section 3).
* ``oracle.mor`` -- O-MOR: the local stage, reduced element, global stage and
  recovery of the MORE-Stress method (section 4).

Every function is pinned by the ``-m "not gpu"`` tests to closed forms,
invariants and the paper's printed values; no function is "parity unpinned".
"""
from . import fem, mor  # noqa: F401
