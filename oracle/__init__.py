"""FP64 CPU oracle for the TaCo query path: test infrastructure only.

Imported by the tests, the smoke check and the benchmark's CPU-baseline leg; never by
the library itself.
"""
from . import taco_oracle  # noqa: F401
