"""Plain, slow, FP64 CPU oracle for the LR-TDDFT response path.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline
leg of the benchmark may import this package.  The product path (the CUDA
library and its Python binding) never imports, links or executes it, and this
package never imports the product; the two share only the seeded input
generator (paper_2510_01875_gb300.workloads), which holds none of the method's
arithmetic.

Every function follows a definition step by step, with library primitives
(LAPACK eigensolver, matrix products, QR) used as single steps and no blocking
or fusion beyond what the definition states:

  crystal.py    empty-core Hamiltonian, plane-wave bases, k-meshes, G-sets
  occupations.py Fermi-Dirac occupations, chemical potential by bisection
  xc.py         ALDA exchange-correlation kernel (Slater + Perdew-Wang 1992)
  response.py   pair densities, Adler-Wiser chi0, Dyson, S(q,w) (Eq. 8),
                F(q,tau) (Eq. 1 with detailed balance), F-tilde (Eq. 2), metrics
  attenuation.py Savitzky-Golay / AICc / constraints filter (Sec. 3, Eqs. 5-7)
  etascan.py    the eta-convergence test in the imaginary-time domain (Sec. 2)
  dielectric.py chi, 1/eps, eps and sigma from a DSF (Kramers-Kronig, Eqs. 10-11)
  kubo.py       the Kubo-Greenwood route to the eta test and the filtered conductivity (App. A.3)
  spectral.py   chi0 through a binned spectral function and its transform (engine variant)
  lindhard.py   continuum finite-temperature Lindhard function (pins only)
  adjoint.py    forward-mode tangents of S(q,w) and F(q,tau) for the gradient pins
  pipeline.py   runs the steps above for one workload

Parity status per function is listed in each module header.
"""
