"""GB300 (sm_103a) modal bispectrum estimator: per-map modal projection, Monte Carlo
linear term and covariance, and the Cholesky-rotated f_NL estimate (Fergusson &
Shellard, arXiv:1105.2791).  The compute runs in the CUDA library built from
csrc/ (see include/modal.h); this package is its ctypes binding."""
from .binding import *  # noqa: F401,F403
from .binding import ModalError, load_library, library_path  # noqa: F401
from .modal import Batch, Plan, ModalBeta, ModalFnl, modal_beta, modal_fnl  # noqa: F401
