"""Oracle: the eta-convergence test in the imaginary-time domain (Sec. 2).

Test infrastructure only (see oracle/__init__.py).

For a list of broadenings eta_1 < eta_2 < ... the whole response path is run once per eta
(pipeline.run_q with the workload's eta replaced), giving per eta the ITCF metrics of Sec. 2:
F(beta/2), int_0^beta F, F~(beta/2), int_0^beta F~ (F~ = F - F(0), Eq. 2) and the static
response.  The paper's rule (Sec. 2, the discussion of its eta-dependence figure): F~(beta/2)
and int F~ converge as eta decreases, and the largest eta within the converged range gives the
reference DSF.  The paper states no numerical criterion; the reading used here:
  eta_j is in the converged range when, for every i <= j and for both F~(beta/2) and
  int_0^beta F~, |m(eta_i) - m(eta_1)| <= tol |m(eta_1)|;
  the reference is the largest such eta_j (eta_1 itself when no other qualifies).
"""
from __future__ import annotations

import numpy as np

from . import pipeline


def metrics_per_eta(wl, etas, iq: int) -> np.ndarray:
    """[n_eta][5] ITCF metrics of q index iq, one full response run per eta."""
    return np.array([pipeline.run_q(wl.replace(eta=float(e)), iq)["metrics"] for e in etas])


def reference_eta(metrics: np.ndarray, tol: float) -> int:
    """Index of the reference eta from metrics [n_eta][5] (etas ascending)."""
    m = np.asarray(metrics)[:, 2:4]          # F~(beta/2), int_0^beta F~
    ref = 0
    for j in range(1, len(m)):
        ok = all(abs(m[i, k] - m[0, k]) <= tol * abs(m[0, k]) for i in range(j + 1) for k in range(2))
        if not ok:
            break
        ref = j
    return ref
