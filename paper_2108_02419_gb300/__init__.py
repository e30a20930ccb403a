"""GB300-native Monte Carlo race rollouts for the BBE sports-betting-exchange model.

Submodules (imported on demand so that importing the package stays light):
  bbe        -- ctypes binding of the C ABI in include/bbe.h (libbbe.so, sm_103a)
  build      -- nvcc build of libbbe.so
  workloads  -- seeded synthetic race-state generators
"""
__all__ = ["bbe", "build", "workloads"]
