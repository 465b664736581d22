"""GB300-native fourth-order AMR elliptic solver (Zhao & Zhang, arXiv 2506.02663).

The compute path is the C-ABI library ``libamr4`` (hand-written sm_103a CUDA kernels) under
``csrc/``; ``amr`` is its thin Python binding.  Importing this package does not load the
library: ``paper_2506_02663_gb300.amr`` does, and it fails loudly when the library is
missing.  ``workloads`` holds the seeded synthetic inputs only.
"""
