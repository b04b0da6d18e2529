"""GB300 (sm_103a) implementation of the self-consistent-field gravity step of
the basis-expansion N-body method for globular-cluster streams (KRIOS II,
arXiv:2602.13385): coefficient reduction, field evaluation, host tidal force
and kick-drift-kick leapfrog as CUDA kernels behind the C ABI of include/scf.h,
and their hand-written adjoint behind ``adjoint.SCFRun`` (torch.autograd).
"""
from .scf import SCF, Config, HOST_HERNQUIST, HOST_MN, HOST_NFW, n_coef, n_lm  # noqa: F401
from . import adjoint  # noqa: F401,E402
