"""GB300-native (sm_103a) compressible-Euler building blocks.

The hot path of FDBB (Moeller & Jaeschke, "FDBB: Fluid Dynamics Building
Blocks"): fused, single-pass, point-wise evaluation of conservative /
primitive / characteristic transforms, the ideal-gas EOS, Riemann invariants,
inviscid fluxes and flux Jacobians over structure-of-arrays fields in GPU
memory.  The CUDA kernels live in ``libfdbb.so`` behind the C ABI of
``include/fdbb.h``; this package is the thin Python binding.

Modules:
  build    -- compile libfdbb.so in-tree (nvcc, sm_103a)
  capi     -- ctypes binding, C names
  blocks   -- torch-tensor wrappers of each entry point
  autograd -- differentiable flux (backward = the flux VJP kernel)
  synth    -- seeded synthetic input fields (no method arithmetic)
"""
from . import build, capi  # noqa: F401

__version__ = "0.1.0"


def __getattr__(name):
    # Tensor wrappers import torch; load them on first use so that the input
    # generators and the build script work without a GPU stack.
    if name in ("blocks", "autograd"):
        import importlib
        return importlib.import_module(__name__ + "." + name)
    raise AttributeError(name)
