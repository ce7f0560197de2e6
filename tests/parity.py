"""Comparison helpers shared by the parity tests.

Per-field error of a GPU state against the oracle's:
  * positive fields (rho, Egas, Erad, kappa): max pointwise |a - b| / |b|
    (|a - b| where b = 0);
  * signed fields (m, F): ||a - b||_inf / ||b||_inf (pointwise relative error
    is meaningless where they cross zero).
"""
import numpy as np

from paper_2404_08247_gb300 import inputs as I

POSITIVE = (I.F_RHO, I.F_EGAS, I.F_ERAD, I.F_KAPPA)


def field_errors(Ug, Uo):
    errs = {}
    for f in range(Uo.shape[0]):
        a = np.asarray(Ug[f], dtype=np.float64)
        b = np.asarray(Uo[f], dtype=np.float64)
        if f in POSITIVE:
            # a field that is zero in the reference (kappa of a gas without
            # coupling) is compared absolutely there
            den = np.where(b != 0.0, np.abs(b), 1.0)
            errs[I.FIELDS[f]] = float(np.max(np.abs(a - b) / den))
        else:
            s = float(np.max(np.abs(b)))
            d = float(np.max(np.abs(a - b)))
            errs[I.FIELDS[f]] = d / s if s > 0 else d
    return errs


def max_error(Ug, Uo):
    return max(field_errors(Ug, Uo).values())


def assert_parity(Ug, Uo, tol, what=""):
    errs = field_errors(Ug, Uo)
    worst = max(errs.values())
    assert worst <= tol, "%s parity %.3e > %.1e: %s" % (what, worst, tol, errs)
    return errs
