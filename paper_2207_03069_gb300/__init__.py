"""GB300-native bulk local search for QUBO (Diverse Adaptive Bulk Search).

The compute path is the C-ABI CUDA library ``libdabs.so`` built from ``csrc/``
for sm_103a; :mod:`paper_2207_03069_gb300.dabs` is its thin ctypes binding.
Instance generators live in :mod:`paper_2207_03069_gb300.workloads`.
"""
__all__ = ["dabs", "workloads"]
