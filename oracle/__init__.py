"""Plain FP64 CPU oracle of the edge-guided densification path.

TEST INFRASTRUCTURE ONLY.  Only tests/, `__graft_entry__.smoke()` and the
`cpu_baseline` / `--impl reference` legs of bench.py may import this package.
The CUDA path (paper_2603_08661_gb300) never imports it, and it imports
nothing from the CUDA path; the two share only the seeded input generators
of `synth`.

* oracle.edge    - edge-importance map, Sec. 2.1 (numpy, FP64)
* oracle.raster  - splatting forward, edge score, adjoint and FD check
                   (C, FP64, oracle/raster.c)
* oracle.densify - top-k selection and Long-Axis-Split, Sec. 2.2 Alg. 1-2
                   (numpy, FP64)

Parity unpinned: none.  Every function is pinned by tests/test_oracle_*.py
against closed forms, library routines (scipy), brute force or invariants.
"""
from . import densify, edge, raster  # noqa: F401
