"""GB300-native dynamic-programming solver for look-ahead eco-driving.

Implements the backward DP sweep and forward rollout of Zhu et al., "A GPU
Implementation of a Look-Ahead Optimal Controller for Eco-Driving Based on
Dynamic Programming" (ECC 2021) as hand-written sm_103a CUDA kernels behind
a C ABI (include/ecodp.h, libecodp.so).

Modules:
  problems  seeded synthetic problem instances (no solver arithmetic)
  native    ctypes binding of libecodp.so (fails loudly if it is not built;
            ECODP_LIBRARY=checked loads the bounds-checked build instead)
  solver    EcoDP, EcoDPBatch, EcoDPValue: PyTorch-facing wrappers (device
            memory, streams, autograd of the adjoint)
  serving   EcoDPServer and the simulated fleet for receding-horizon re-solves
  build     nvcc build of libecodp.so and libecodp_checked.so
"""

__all__ = ["EcoDP", "problems"]


def __getattr__(name):
    if name == "EcoDP":
        from .solver import EcoDP
        return EcoDP
    raise AttributeError(name)
