"""GB300-native Benelux-pair search (arXiv 2506.01099).

The compute lives in ``libbenelux.so`` (hand-written sm_103a CUDA behind a C
ABI, declared in ``include/benelux.h``).  ``paper_2506_01099_gb300.benelux``
is the thin ctypes binding; ``workloads`` holds the seeded input generators.
Nothing is imported eagerly so that the input generators can be used on a
machine without the built library.
"""

__all__ = ["benelux", "workloads", "build"]
