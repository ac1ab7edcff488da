"""GB300-native hot path of VSA-OGM (arXiv 2408.09066).

The computation runs in hand-written sm_103a CUDA kernels behind the C ABI
declared in ``include/vsaogm.h`` (``libvsaogm.so``).  ``vsaogm`` is the thin
ctypes binding; ``synth`` generates seeded synthetic lidar inputs.  Importing
this package loads nothing: the library is opened on first use of the binding,
and fails loudly if it has not been built.
"""
