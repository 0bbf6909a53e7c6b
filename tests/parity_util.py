"""Error measures shared by the GPU parity tests.

Every comparison reports two numbers against the oracle's array `want`:
  rel  = ||got - want||_2 / ||want||_2          (field-wide relative L2)
  max  = max |got - want| / max |want|          (worst element, relative to
                                                 the field's largest entry)
so an error confined to a few elements (a wrong wall node, one bad row of a
large box) cannot hide under the field-wide norm.  `check` prints both with
a tag (run pytest with -s to see them) and asserts each against its bar.
"""
import os

import numpy as np


def tid():
    """Name of the running test (with its parameters), for the printed tags."""
    return os.environ.get("PYTEST_CURRENT_TEST", "?").split("::")[-1].split(" ")[0]


def errs(got, want):
    got = np.asarray(got, dtype=np.float64).ravel()
    want = np.asarray(want, dtype=np.float64).ravel()
    d = got - want
    nw = max(float(np.linalg.norm(want)), 1e-300)
    mw = max(float(np.abs(want).max()) if want.size else 0.0, 1e-300)
    r = float(np.linalg.norm(d)) / nw
    m = float(np.abs(d).max()) / mw if d.size else 0.0
    return r, m


def check(tag, got, want, rel_tol, max_tol):
    r, m = errs(got, want)
    print("PARITY %-48s rel %.2e (bar %.0e)  max %.2e (bar %.0e)" % (tag, r, rel_tol, m, max_tol))
    assert r < rel_tol, (tag, "rel", r, rel_tol)
    assert m < max_tol, (tag, "max", m, max_tol)
    return r, m


def pos_err(a, b, shape):
    """Largest periodic-image distance between two position arrays."""
    d = np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64)
    Lb = np.array(shape, dtype=np.float64)
    d -= Lb * np.round(d / Lb)
    return float(np.abs(d).max()) if d.size else 0.0


def check_pos(tag, a, b, shape, tol):
    e = pos_err(a, b, shape)
    print("PARITY %-48s pos %.2e (bar %.0e)" % (tag, e, tol))
    assert e < tol, (tag, "pos", e, tol)
    return e
