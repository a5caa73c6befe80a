"""GB300 (sm_103a) reduction-reuse row kernels with DSMEM cluster staging.

``credit``  ctypes binding of libcredit.so (the C ABI in include/credit.h)
``build``   nvcc build of libcredit.so, in-tree
``synth``   seeded synthetic inputs
"""
__all__ = ["credit", "build", "synth"]
