"""CPU oracle for the Clenshaw-Curtis spherical-harmonic transform.

TEST INFRASTRUCTURE.  This package is a plain, slow, obviously correct CPU
restatement of Hotta & Ujiie (2018), "A nestable, multigrid-friendly grid on
a sphere for global spectral models based on Clenshaw-Curtis quadrature".
Only the tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  The GPU library
never imports, links or calls anything here, and nothing here imports the
GPU library: the two share no code.

Contents (all FP64 except the binary128 Legendre recurrence of Sec. 4.1):

* ``cc_nodes``, ``cc_weights``     -- Eq. (cc-points), Eq. (cc-wgt)
* ``fejer1_nodes``, ``fejer1_weights``, ``analysis_fejer1``,
  ``synthesis_fejer1``             -- the shifted grid of Fejer's first
                                      rule, Sec. 3.3 (Eq. fejer1-points and
                                      the interpolatory form of Eq. fejer1-wgt)
* ``gauss_nodes_weights``          -- Eq. (gauss-quad)/(gauss-wgt) by the
                                      Golub-Welsch eigenproblem
* ``pnm_cc``, ``pnm_at``           -- P~_n^m by the recurrence in binary128
* ``dft_forward``, ``dft_inverse`` -- Eq. (dFT) discretised, and its inverse
* ``analysis``, ``synthesis``      -- Eq. (dSHT)/(cc-quad), Eq. (iSHT)/(iLT)
* ``adjoint_analysis``, ``adjoint_synthesis`` -- transposes of the two
  (``adjoint_analysis_rows`` and ``adjoint_synthesis(..., ms=...)``
  evaluate them at chosen latitudes or zonal wavenumbers only)
* ``synthesis_rows``               -- Eq. (iSHT) at chosen latitudes
* ``restrict_nested``              -- Sec. 3.2 / Appendix C
* ``reduced_sizes``, ``analysis_reduced``, ``synthesis_reduced`` -- reduced
                                      Clenshaw-Curtis grids with per-latitude
                                      longitude counts (the reduction rule
                                      quoted in Sec. 6)
"""
from .cc_oracle import *  # noqa: F401,F403
from .cc_oracle import __all__  # noqa: F401
