"""GB300 (sm_103a) discrete-ordinates CT dose solver.

Implements the data-parallel hot path of Norris & Liu, arXiv:1811.12391:
Siddon ray tracing of the uncollided fluence and its first-collision source
(Sec. II.A), step-differenced octant wavefront sweeps of the collided
multigroup problem (Eq. 2) with Legendre-moment scattering, the scalar
fluence (Eq. 3) and the dose tally, plus the discrete adjoint.  The compute
runs in libdoctors.so (CUDA, C-ABI in include/doctors.h); this package only
marshals arguments and uses PyTorch for device memory and streams.
"""
from . import _lib  # noqa: F401
from ._lib import DoctorsError  # noqa: F401

__all__ = ["DoctorsError", "DoctorsProblem", "quadrature"]


def __getattr__(name):
    if name in ("DoctorsProblem", "quadrature"):
        from . import solver
        return getattr(solver, name)
    raise AttributeError(name)
