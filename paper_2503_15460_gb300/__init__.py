"""GB300 tree-tensor-network (ML-MCTDH) projector-splitting time evolution.

The compute path is the CUDA library ``libttn.so`` (C ABI in include/ttn.h);
``paper_2503_15460_gb300.ttn`` is its ctypes binding and
``paper_2503_15460_gb300.build`` compiles it.  Importing this package does not
load the library; importing ``.ttn`` does, and fails if it is not built.
"""
