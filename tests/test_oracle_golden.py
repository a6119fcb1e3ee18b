"""The oracle against its stored result on the small workload (l_max = 32, 33 x 128 grid,
6 modes, seed 0): beta_n, alpha_n of the local shape and the fNL estimate with sigma from
the closed-form zeta.  The file was written by tests/golden/make_tiny.py from the oracle
itself, so this guards against unintended changes of the oracle's arithmetic; a change
made on purpose regenerates the file in the same commit, naming the passage behind it."""
import importlib.util
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _maker():
    spec = importlib.util.spec_from_file_location("make_tiny", os.path.join(HERE, "golden", "make_tiny.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_small_workload_matches_the_stored_oracle_result():
    mk = _maker()
    beta0, alpha0, fnl0, sigma0, modes = mk.read(os.path.join(HERE, "golden", mk.NAME))
    from oracle import modal as om
    assert [tuple(m) for m in modes] == list(om.mode_list(6))
    beta, alpha, fnl, sigma = mk.compute()
    assert np.linalg.norm(beta - beta0) <= 1e-10 * np.linalg.norm(beta0)
    assert np.linalg.norm(alpha - alpha0) <= 1e-10 * np.linalg.norm(alpha0)
    assert fnl == pytest.approx(fnl0, rel=1e-8, abs=1e-12 * sigma0)
    assert sigma == pytest.approx(sigma0, rel=1e-10)
    # a Gaussian map: the local-shape estimate is consistent with zero
    assert abs(fnl0) < 5 * sigma0
