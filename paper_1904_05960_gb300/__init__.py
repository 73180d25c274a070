"""GB300-native multigrid-reduction (MGR) preconditioned flexible GMRES for
multiphase poromechanics Jacobians.

Submodules:
  mgr    -- ctypes binding of the C ABI in include/mgr_gb300.h (libmgr_gb300.so)
  build  -- in-tree nvcc build of the CUDA library for sm_103a
  synth  -- seeded synthetic Jacobians (input generator; no solver arithmetic)

Importing the package does not load the CUDA library; ``mgr.lib()`` does.
"""
__all__ = ["mgr", "build", "synth"]
