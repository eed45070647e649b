"""CPU FP64 oracle for the directional scale-discretized wavelet transform.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, links or
executes this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.

The oracle is the plain definition of what the GPU path computes, written out
as direct sums in float64 (McEwen, Vandergheynst & Wiaux, "On the computation
of directional scale-discretized wavelet transforms on the sphere", 2013):

* kernels: Sec. 2.2, Eqs. (7), (11)-(16);
* sampling and quadrature: Sec. 3.1, Eqs. (17)-(19) and the SO(3) grid;
* analysis: Sec. 3.2, Eq. (20) (harmonic form of Eq. (1)) and the scaling
  coefficients of Eq. (3);
* synthesis: Sec. 3.3, Eqs. (32)-(33) and (41), with every integral replaced
  by the exact quadrature of Sec. 3.1.

It shares no code with the CUDA path.  Parity status of every function is
listed in ``s2dw_oracle.PARITY``.
"""
from .s2dw_oracle import *  # noqa: F401,F403
from .s2dw_oracle import __all__  # noqa: F401
