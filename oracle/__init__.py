"""FP64 CPU oracle (test infrastructure only; see oracle/estimator.py)."""
from .sph import wigner3j, ylm, legendre, n_lll, h_lll, allowed_multipole  # noqa: F401
from . import estimator  # noqa: F401
