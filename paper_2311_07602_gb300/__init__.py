"""lrbatch: batched small/rectangular FP64 GEMM for GB300 (sm_103a).

The compute lives in the CUDA shared library built from csrc/; `lrbatch`
(this package's binding module) marshals arguments to its C ABI.  Importing
the package loads nothing; the library is opened on first use and raises if
it is missing.
"""
