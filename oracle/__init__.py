"""FP64 CPU oracle for the discrete-ordinates CT dose hot path.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of what Norris & Liu (arXiv:1811.12391) compute: level-symmetric
S_N quadrature (Sec. II.D), Legendre-moment scattering (Eq. 2), Siddon ray
tracing of the uncollided fluence and the first-collision source (Sec. II.A),
step- or diamond-differenced transport sweeps with vacuum boundaries (Eq. 2),
source iteration, the quadrature sum for the scalar fluence (Eq. 3), the dose
tally, and the CT-number to material conversion of the input (Sec. II.B).  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import it; the product path (``paper_1811_12391_gb300``)
never does, and the two share no code.

Modules:
  quadrature  level-symmetric directions/weights, real spherical harmonics
  transport   ctypes binding of transport.c (Siddon walks, sweep)
  solver      uncollided fluence, source iteration, dose, adjoint, gradients
  ct          CT numbers -> materials and densities (piecewise calibration)
"""
