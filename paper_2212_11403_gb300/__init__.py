"""GB300-native Li & Stephens all-vs-all hot path (arXiv 2212.11403, kalis).

The compute path is the C-ABI library ``libls`` (CUDA kernels for sm_103a, declared in
``include/ls.h``); ``paper_2212_11403_gb300.ls`` is its thin ctypes binding and
``paper_2212_11403_gb300.synth`` draws the seeded synthetic workloads.  Importing this package
does not load the library; ``paper_2212_11403_gb300.ls`` does, and fails loudly if it is missing.
"""

__all__ = ["ls", "synth"]
