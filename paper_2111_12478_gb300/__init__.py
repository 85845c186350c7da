"""GWCP predictive race analysis on GB300 (sm_103a).

The hot path (trace decode, epoch assignment, critical-section annotation, clock
propagation, access grouping, per-address check, race compaction) runs in the CUDA
library ``libgwcp.so`` built from ``csrc/``; ``gwcp`` is its thin ctypes binding.
"""
