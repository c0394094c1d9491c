"""FP64 CPU oracle for the PRISM fit -- test infrastructure only.

Imported only by tests, the smoke check and the benchmark's CPU-baseline leg.
It shares no code with the CUDA library and never imports the package.
"""
from . import prism_oracle, metrics, slabs  # noqa: F401
