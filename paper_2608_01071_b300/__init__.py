"""B300-native lattice kinetic scheme with grid-separated moving rigid bodies and its exact discrete adjoint.

The compute path is the CUDA library ``liblks.so`` (C ABI in ``include/lks.h``); this package only
marshals arguments.  ``Solver`` wraps one library context; ``LKSFunction`` exposes forward/adjoint to
torch.autograd.
"""
from .binding import Batch, LKSError, Solver, params_from_workload  # noqa: F401

__all__ = ["Solver", "Batch", "LKSError", "params_from_workload"]
