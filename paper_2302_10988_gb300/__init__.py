"""GB300-native (sm_103a) ALI-FMM travel times, ray paths and adjoint gradients.

The compute path is the C-ABI library ``libalifmm.so`` built from ``csrc/``; the
Python modules here only marshal arguments (``binding``) and generate seeded
synthetic inputs (``workloads``).  Importing the package does not load the
library; the binding loads it on first use and fails loudly when it is missing.
"""
__all__ = ["binding", "workloads", "api"]
