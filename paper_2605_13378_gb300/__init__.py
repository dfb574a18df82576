"""GB300 (sm_103a) Jacobian-free Newton-Krylov hot path with AD and FD Jacobian-vector products.

The compute path is the C-ABI library ``libjfnk.so`` (declared in
include/jfnk.h, built from csrc/ by ``build.py``); ``paper_2605_13378_gb300.jfnk``
is its Python binding. Importing the package does not load the library;
importing ``paper_2605_13378_gb300.jfnk`` does, and fails loudly when it has
not been built.
"""
__all__ = ["build", "jfnk"]
