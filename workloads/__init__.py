"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package generates circuits (gate lists) and initial site tensors.  It holds
none of the method's arithmetic: no contraction, no decomposition, no truncation.
Both the CPU oracle and the GPU library consume what it produces.
"""

from . import gates, circuits, states  # noqa: F401
