"""GB300 multi-key TFHE gate bootstrapping (arXiv 2205.05825).

The compute path is the CUDA library ``libmktfhe.so`` (C ABI in
include/mk_tfhe.h); ``binding`` is its thin ctypes binding, ``workloads`` the
seeded synthetic inputs, ``serving`` the request-serving front end and
``regression`` the encrypted linear-regression application built on the
library's k-bit operators.  Importing this package does not load the
library; ``binding.load()`` does, and fails loudly if it has not been built.
"""
__all__ = ["binding", "workloads", "build", "serving", "regression"]
