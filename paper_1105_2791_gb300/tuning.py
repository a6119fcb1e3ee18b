"""Cache of autotuned launch shapes (modal_autotune), one JSON file per user.

The library's autotuner (include/modal.h: modal_autotune) times candidate launch shapes of
a plan on the caller's maps; this module keys the winner by everything that decides
which shape wins (device name, l_max, P, grid, precision, batch size, linear-term mode)
and stores it in a JSON object {key: {"chunk", "legendre_maps", "cubic_ctas", "ms"}}, so
that later plans of the same configuration take the tuned shapes without timing.  Host-side bookkeeping only: no part of the method runs here.
"""
from __future__ import annotations

import json
import os
import tempfile

from . import binding as B

PREC_NAMES = {v: k for k, v in B.PREC.items()}


def tuning_key(device, lmax, P, nrings, nphi, prec, batch, use_linear, linear_mode, masked):
    """The cache key of one configuration (a plain string, stable across runs)."""
    prec_name = PREC_NAMES.get(prec, str(prec))
    return "%s|lmax=%d|P=%d|grid=%dx%d|%s|B=%d|linear=%s|mask=%d" % (
        device, lmax, P, nrings, nphi, prec_name, batch, linear_mode if use_linear else "off", int(bool(masked)))


def load(path):
    """The cache as a dict ({} if the file does not exist)."""
    if not path or not os.path.exists(path):
        return {}
    with open(path) as f:
        data = json.load(f)
    if not isinstance(data, dict):
        raise ValueError("tuning cache %s is not a JSON object" % path)
    return data


def store(path, key, tuning):
    """Add or replace one entry; the file is rewritten atomically (temporary file + rename)."""
    data = load(path)
    data[key] = {k: (float(tuning[k]) if k == "ms" else int(tuning[k]))
                 for k in B.TUNING_FIELDS + ("ms",) if k in tuning}
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(prefix=".tuning.", dir=d)
    try:
        with os.fdopen(fd, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
            f.write("\n")
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.unlink(tmp)
        raise


def valid_entry(entry):
    """True if a cached entry carries every field modal_set_tuning needs, as positive ints."""
    try:
        return all(int(entry[k]) >= 1 for k in B.TUNING_FIELDS)
    except (KeyError, TypeError, ValueError):
        return False
