"""GB300-native wave path tracer for holography (sm_103a CUDA library + thin Python binding).

``scenes`` makes seeded synthetic inputs; ``hpt`` binds the C-ABI of ``include/hpt.h``;
``build`` compiles the CUDA library in-tree.  Importing the package does not load the
library; ``hpt.load_library()`` does, and fails loudly when it is missing.
"""
