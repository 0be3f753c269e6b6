"""B300-native McMg online solve: FGMRES on the heterogeneous Helmholtz
operator, preconditioned by the multi-channel multigrid V-cycle, in
hand-written sm_103a CUDA behind a C ABI (``include/mcmg.h``).

``mcmg`` is the ctypes binding to the in-tree shared library; ``inputs``
draws the seeded synthetic workloads.
"""
