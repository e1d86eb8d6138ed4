"""FP64 CPU oracle of the Allegro-FM energy/force hot path (arXiv 2502.06073).

TEST INFRASTRUCTURE ONLY.  This package is the independent, plain definition that the
CUDA path is checked against.  Only the test suite, the package smoke check and the
benchmark's CPU-baseline leg may import it; the library never does, and the two share
no code (the synthetic inputs come from the separate `synth` package).

Modules: so3 (spherical harmonics, coupling tensors, paths), weights (SplitMix64 init),
neighbors (brute-force float32-predicate edge lists), allegro64 (energy + hand-derived
gradient), md (velocity Verlet).

Parity status: every function here is pinned by tests/test_oracle_*.py (closed forms,
invariances, finite differences, brute-force/library cross-checks).  One item is
"parity unpinned": the accuracy of a trained model (no weights or data exist).
"""
from .allegro64 import Allegro64  # noqa: F401
from . import so3, weights, neighbors, md, pool  # noqa: F401
