"""GB300-native nested block preconditioned solver for the VMS Navier-Stokes
tangent [[A, B], [C, D]] (Liu, Yang, Dong & Marsden, arXiv:1911.10814).

The method runs in libnbp.so (hand-written sm_103a CUDA, C ABI in
include/nbp.h); ``nbp`` is its ctypes binding and ``autograd`` the
torch.autograd.Function around the solve and its adjoint.
"""
from . import build  # noqa: F401
from .nbp import BatchSolver, Solver, Vms, default_options, load, NbpError, rcr_step  # noqa: F401
