"""Plain FP64 CPU oracle for the Fisher-BT hot path (Hong, Abdulah, Genton & Sun, arXiv 2601.11437).

TEST INFRASTRUCTURE ONLY.  Only tests, the package smoke check and the bench's CPU-baseline leg may
import or run anything here; the product path (the CUDA library and its Python binding) never does.
It shares no code with the CUDA path: its inputs come from the caller (the seeded generators) and
its arithmetic is written here from the paper's definitions, slowly and plainly.

Modules
  special        K_nu(x) and dK_nu/dnu by trapezoid quadrature of their integral representations
                 (DLMF 10.32.9 and its nu-derivative), digamma (asymptotic series + recurrence).
  paper_series   Supplementary A of the paper: the five-case evaluation of d/dnu[x^nu K_nu(x)]
                 (small-x series, Debye uniform expansion with the U_k recursion, Hankel expansion).
  matern         Matern covariance C(h; theta) (Sec. 2.1) and its partials in sigma^2, alpha (Sec. 2.2)
                 and nu (Sec. 2.2 + Supp. A); dense Sigma, Sigma_alpha, Sigma_nu.
  linalg         textbook blocked Cholesky, forward / back substitution, log-determinant.
  likelihood     Algorithm 2 (log-likelihood) and Algorithm 3 (log-likelihood, score, Fisher
                 information), Eq. 1-4.
  fisher_bt      Algorithm 1 (Fisher scoring with the relaxed Armijo backtracking line search,
                 Eq. 5), the L9 initial design (Table 1), the call-count shift rule and the
                 Nelder-Mead fallback (Sec. 2.1).
  fields         z = L_true e for seeded synthetic fields, and the script writing stored fields.

Parity status: every function has a pin in tests/test_oracle_*.py (closed forms, library routines,
brute force in extended precision, finite differences, invariances).  Nothing here is "parity
unpinned" except what the paper prints for its soil-moisture data (Table 2), which needs a dataset
that is not available; no function here reproduces it.
"""
from . import special, paper_series, matern, linalg, likelihood, fisher_bt, fields  # noqa: F401
