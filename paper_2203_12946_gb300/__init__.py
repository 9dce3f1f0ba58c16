"""GB300 (sm_103a) implementation of the essentially entropic lattice Boltzmann
step of Atif, Kolluru & Ansumali (arXiv:2203.12946).

The compute path is the CUDA library ``libelbm.so`` (C ABI in
``include/elbm.h``); ``paper_2203_12946_gb300.elbm`` is its thin Python binding
and ``paper_2203_12946_gb300.inputs`` the seeded synthetic inputs.  Importing
this package does not load the library; the first call that needs it does,
and raises if it is missing.
"""

__all__ = ["elbm", "inputs", "build"]
